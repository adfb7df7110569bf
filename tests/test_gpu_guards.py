"""Outputs are written exactly where they belong: every output vector and
matrix is a view into a larger buffer filled with a sentinel, at ragged
sizes (tails of strips, row groups and 16-byte chunks), and after each call
the sentinel regions around it are unchanged, while the results themselves
match the FP64 oracle."""

import numpy as np
import pytest
import torch

import oracle
from gpu_util import ALPHA, BETA, U, built, dev, host  # noqa: F401
from tolerance import check_reduce

pytestmark = pytest.mark.gpu

SENT = 12345.0
PAD = 64  # floats of guard on each side (keeps the view 16-byte aligned)


def guarded(n):
    """A length-n view in the middle of a sentinel-filled buffer."""
    buf = torch.full((n + 2 * PAD,), SENT, device=dev())
    return buf, buf[PAD:PAD + n]


def guarded_mat(m, n, extra_cols=5):
    """An m x n view (row stride n + extra_cols) inside a sentinel buffer."""
    ld = n + extra_cols
    buf = torch.full(((m + 2) * ld + 2 * PAD,), SENT, device=dev())
    view = buf[PAD + ld:PAD + ld + m * ld].view(m, ld)[:, :n]
    return buf, view


def untouched(buf, view):
    """Every element of buf outside view still holds the sentinel."""
    mask = torch.ones(buf.numel(), dtype=torch.bool, device=dev())
    base = view.storage_offset() - buf.storage_offset()
    if view.dim() == 1:
        mask[base:base + view.numel()] = False
    else:
        m, n = view.shape
        ld = view.stride(0)
        for i in range(m):
            mask[base + i * ld:base + i * ld + n] = False
    torch.cuda.synchronize()
    return bool(torch.all(buf[mask] == SENT))


@pytest.mark.parametrize("m,n", [(1, 1), (37, 1029), (1031, 517), (2051, 4099)])
def test_bicgk_and_gesummv_write_only_their_outputs(built, m, n):
    kf = built
    A, B, p, r = U((m, n), 1), U((m, n), 2), U((n,), 3), U((m,), 4)
    bq, q = guarded(m)
    bs, s = guarded(n)
    kf.kf_bicgk(A, p, r, q, s, kf.workspace(kf.KF_SEQ_BICGK, m, n))
    assert untouched(bq, q) and untouched(bs, s)
    Ah, ph, rh = host(A), host(p), host(r)
    qo, so = oracle.bicgk(Ah, ph, rh)
    check_reduce(host(q), qo, oracle.abs_gemv(Ah, ph), n, "q")
    check_reduce(host(s), so, oracle.abs_gemvt(Ah, rh), m, "s")
    by, y = guarded(m)
    kf.kf_gesummv(A, B, p, ALPHA, BETA, y, kf.workspace(kf.KF_SEQ_GESUMMV, m, n))
    assert untouched(by, y)
    yo = oracle.gesummv(Ah, host(B), ph, ALPHA, BETA)
    check_reduce(host(y), yo, ALPHA * oracle.abs_gemv(Ah, ph) + BETA * oracle.abs_gemv(host(B), ph), n, "y")


@pytest.mark.parametrize("n", [9, 1030, 2053])
def test_gemver_writes_only_its_outputs(built, n):
    kf = built
    A = U((n, n), 1)
    vs = [U((n,), t) for t in (5, 6, 7, 8, 4, 9)]
    bB, B = guarded_mat(n, n)
    bx, x = guarded(n)
    bw, w = guarded(n)
    kf.kf_gemver(A, *vs, ALPHA, BETA, B, x, w, kf.workspace(kf.KF_SEQ_GEMVER, n, n))
    assert untouched(bB, B) and untouched(bx, x) and untouched(bw, w)
    Bo, xo, wo = oracle.gemver(host(A), *[host(v) for v in vs], ALPHA, BETA)
    assert np.max(np.abs(host(B) - Bo)) <= 4 * 2.0 ** -24 * 4.0 * (1 + np.max(np.abs(Bo)))


@pytest.mark.parametrize("n", [8, 1028, 4100])
def test_gemver_single_launch_writes_only_its_outputs(built, n):
    kf = built
    A = U((n, n), 1)
    vs = [U((n,), t) for t in (5, 6, 7, 8, 4, 9)]
    buf = torch.full((n * (n + 4) + 2 * PAD,), SENT, device=dev())
    B = buf[PAD:PAD + n * (n + 4)].view(n, n + 4)[:, :n]      # ldb = n + 4 keeps rows 16-byte aligned
    bx, x = guarded(n)
    bw, w = guarded(n)
    kf.kf_gemver_single(A, *vs, ALPHA, BETA, B, x, w, kf.workspace(kf.KF_SEQ_GEMVER, n, n))
    assert untouched(buf, B) and untouched(bx, x) and untouched(bw, w)
    Bo, xo, wo = oracle.gemver(host(A), *[host(v) for v in vs], ALPHA, BETA)
    sx = BETA * oracle.abs_gemvt(Bo, host(vs[4])) + np.abs(host(vs[5]))
    check_reduce(host(x), xo, sx, n, "x")


@pytest.mark.parametrize("m,n", [(5, 8), (1003, 2052), (4097, 1028)])
def test_atax_and_sgemvt_write_only_their_outputs(built, m, n):
    kf = built
    A, x0, y0, z0 = U((m, n), 1), U((n,), 3), U((m,), 4), U((n,), 9)
    by, y = guarded(n)
    kf.kf_atax(A, x0, y, kf.workspace(kf.KF_SEQ_ATAX, m, n))
    assert untouched(by, y)
    Ah, xh = host(A), host(x0)
    check_reduce(host(y), oracle.atax(Ah, xh)[0], oracle.abs_gemvt(Ah, oracle.abs_gemv(Ah, xh)), max(m, n), "y")
    bx, x = guarded(n)
    bw, w = guarded(m)
    kf.kf_sgemvt(A, y0, z0, ALPHA, BETA, x, w, kf.workspace(kf.KF_SEQ_SGEMVT, m, n))
    assert untouched(bx, x) and untouched(bw, w)
    if m >= 8 and n % 4 == 0:   # the single launch's rule
        bx, x = guarded(n)
        bw, w = guarded(m)
        kf.kf_sgemvt_single(A, y0, z0, ALPHA, BETA, x, w, kf.workspace(kf.KF_SEQ_SGEMVT, m, n))
        assert untouched(bx, x) and untouched(bw, w)
        xo, wo = oracle.sgemvt(Ah, host(y0), host(z0), ALPHA, BETA)
        sx = BETA * oracle.abs_gemvt(Ah, host(y0)) + np.abs(host(z0))
        check_reduce(host(x), xo, sx, m, "x")
        check_reduce(host(w), wo, ALPHA * oracle.abs_gemv(Ah, np.abs(xo) + sx), max(m, n), "w")


@pytest.mark.parametrize("n", [1, 3, 1027, (1 << 20) + 5])
def test_vector_passes_write_only_their_outputs(built, n):
    kf = built
    w0, v0, u0 = U((n,), 10), U((n,), 11), U((n,), 12)
    bz, z = guarded(n)
    br, r = guarded(1)
    kf.kf_axpydot(w0, v0, u0, ALPHA, z, r, kf.workspace(kf.KF_SEQ_AXPYDOT, 1, n))
    assert untouched(bz, z) and untouched(br, r)
    zo, ro = oracle.axpydot(host(w0), host(v0), host(u0), ALPHA)
    assert abs(float(host(r)[0]) - ro) <= 1e-5 * np.sqrt(n) * float(np.sum(np.abs(zo * host(u0))))
    bo, o = guarded(n)
    kf.kf_waxpby(ALPHA, w0, BETA, v0, o)
    assert untouched(bo, o)
