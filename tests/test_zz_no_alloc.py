"""kf_bicgk_noalloc: BiCGK for callers that cannot allocate device memory.

Such callers (a framework that forbids allocation while it records work, a
host whose device memory belongs to another allocator, a plain C program
with no device allocator) cannot provide the workspace kf_bicgk needs;
kf_bicgk_noalloc uses a fixed scratch array inside the library instead.

These tests call it through the C ABI twice in a row, with different inputs,
and check each result against the FP64 oracle (relative 1e-5 sqrt(reduction
length), normwise and componentwise) and against kf_bicgk's result on the
same inputs within the same tolerance.  The second call catches state left
over from the first (the array keeps it).  They also check that a call
allocates no device memory, that a bulk-copy tuning fixed by the user still
gives correct results (the call takes the direct-load form), the empty
cases, and the largest square shape the array holds.

The file is named so that pytest collects it last.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import built, dev, host  # noqa: F401
from tolerance import check_reduce, rel_tol

pytestmark = pytest.mark.gpu


def _call(L, A, p, r, q, s):
    m, n = A.shape
    stream = torch.cuda.current_stream().cuda_stream
    return L.kf_bicgk_noalloc(m, n, A.data_ptr(), A.stride(0), p.data_ptr(), r.data_ptr(), q.data_ptr(),
                              s.data_ptr(), stream)


def _inputs(m, n, seed):
    A = synth.uniform((m, n), seed, synth.TID["A"], device=dev())
    p = synth.uniform((n,), seed, synth.TID["p"], device=dev())
    r = synth.uniform((m,), seed, synth.TID["r"], device=dev())
    return A, p, r


def _check(kf, L, m, n, seed, what):
    A, p, r = _inputs(m, n, seed)
    q = torch.full((m,), float("nan"), device=dev())
    s = torch.full((n,), float("nan"), device=dev())
    st = _call(L, A, p, r, q, s)
    assert st == 0, L.kf_last_error()
    Ah, ph, rh = host(A), host(p), host(r)
    qo, so = oracle.bicgk(Ah, ph, rh)
    check_reduce(host(q), qo, np.abs(Ah) @ np.abs(ph), n, f"q vs oracle, {what}")
    check_reduce(host(s), so, np.abs(Ah).T @ np.abs(rh), m, f"s vs oracle, {what}")
    # and against the entry point with a workspace, on the same inputs
    q0, s0 = torch.empty(m, device=dev()), torch.empty(n, device=dev())
    kf.kf_bicgk(A, p, r, q0, s0, kf.workspace(kf.KF_SEQ_BICGK, m, n))
    tq, ts = rel_tol(n), rel_tol(m)
    assert np.max(np.abs(host(q) - host(q0))) <= tq * max(np.max(np.abs(qo)), 1e-300), what
    assert np.max(np.abs(host(s) - host(s0))) <= ts * max(np.max(np.abs(so)), 1e-300), what


@pytest.mark.parametrize("m,n", [(3000, 2500), (1031, 777)])
def test_noalloc_two_calls_match_the_oracle(built, m, n):
    kf = built
    L = kf.lib()
    for call, seed in enumerate((11, 12)):
        _check(kf, L, m, n, seed, f"{m}x{n}, call {call + 1}")


def test_noalloc_allocates_nothing(built):
    """After a first call (which loads the module and looks up the array),
    a second call changes the device's free memory by nothing."""
    kf = built
    L = kf.lib()
    m, n = 2048, 1536
    A, p, r = _inputs(m, n, 21)
    q, s = torch.empty(m, device=dev()), torch.empty(n, device=dev())
    assert _call(L, A, p, r, q, s) == 0, L.kf_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _call(L, A, p, r, q, s) == 0, L.kf_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_with_a_fixed_bulk_copy_tuning(built):
    """A tuning fixed with a bulk-copy ring depth: kf_bicgk takes the staged
    form, kf_bicgk_noalloc the direct form of the same shape; both match
    the oracle, on two calls in a row."""
    kf = built
    L = kf.lib()
    kf.kf_set_matrix_tuning(8, 1, 4, 0, 3)
    try:
        for call, seed in enumerate((31, 32)):
            _check(kf, L, 2100, 3000, seed, f"staged tuning fixed, call {call + 1}")
    finally:
        kf.kf_set_matrix_tuning(0, 0, 0, 0, 0)


def test_noalloc_largest_square_that_fits(built):
    kf = built
    L = kf.lib()
    _check(kf, L, 8192, 8192, 41, "8192x8192")


@pytest.mark.parametrize("m,n", [(0, 300), (300, 0)])
def test_noalloc_empty_side(built, m, n):
    """An empty side gives an empty sum: the other output is all zeros."""
    kf = built
    L = kf.lib()
    A = torch.zeros((max(m, 1), max(n, 1)), device=dev())[:m, :n]
    p = torch.ones(n, device=dev())
    r = torch.ones(m, device=dev())
    q = torch.full((m,), float("nan"), device=dev())
    s = torch.full((n,), float("nan"), device=dev())
    stream = torch.cuda.current_stream().cuda_stream
    st = L.kf_bicgk_noalloc(m, n, A.data_ptr(), max(n, 1), p.data_ptr() if n else None,
                            r.data_ptr() if m else None, q.data_ptr() if m else None,
                            s.data_ptr() if n else None, stream)
    assert st == 0, L.kf_last_error()
    torch.cuda.synchronize()
    assert torch.all(q == 0) and torch.all(s == 0)


def test_noalloc_rejects_shapes_beyond_the_scratch(built):
    kf = built
    L = kf.lib()
    big = 1 << 15
    st = L.kf_bicgk_noalloc(big, big, 256, big, 256, 256, 256, 256, None)
    assert st == -2
    assert b"bytes of scratch" in L.kf_last_error()
