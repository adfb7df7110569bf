"""kf_bicgk_noalloc: BiCGK for callers that cannot allocate device memory.

Such callers (a framework that forbids allocation while it records work, a
host whose device memory belongs to another allocator, a plain C program)
cannot provide the workspace kf_bicgk needs; kf_bicgk_noalloc uses a fixed
scratch array inside the library instead.  This test calls it through the C
ABI twice in a row, with different inputs, and checks each result against
kf_bicgk's on the same inputs with the tolerance of the other parity tests
(relative 1e-5 sqrt(reduction length), normwise and componentwise).  The
second call catches state left over from the first (the array keeps it).

The file is named so that pytest collects it last.
"""

import numpy as np
import pytest
import torch

import synth
from gpu_util import built, dev, host  # noqa: F401
from tolerance import check_reduce

pytestmark = pytest.mark.gpu


def _abs_gemv(A, x):
    return np.abs(A) @ np.abs(x)


def _abs_gemvt(A, y):
    return np.abs(A).T @ np.abs(y)


@pytest.mark.parametrize("m,n", [(3000, 2500), (1031, 777)])
def test_noalloc_matches_workspace_entry_point(built, m, n):
    kf = built
    L = kf.lib()
    ws = kf.workspace(kf.KF_SEQ_BICGK, m, n)
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((11, 12)):
        A = synth.uniform((m, n), seed, synth.TID["A"], device=dev())
        p = synth.uniform((n,), seed, synth.TID["p"], device=dev())
        r = synth.uniform((m,), seed, synth.TID["r"], device=dev())
        q0 = torch.empty(m, device=dev()); s0 = torch.empty(n, device=dev())
        kf.kf_bicgk(A, p, r, q0, s0, ws)
        q = torch.full((m,), float("nan"), device=dev()); s = torch.full((n,), float("nan"), device=dev())
        st = L.kf_bicgk_noalloc(m, n, A.data_ptr(), A.stride(0), p.data_ptr(), r.data_ptr(),
                                q.data_ptr(), s.data_ptr(), stream)
        assert st == 0, L.kf_last_error()
        Ah, ph, rh = host(A), host(p), host(r)
        check_reduce(host(q), host(q0), _abs_gemv(Ah, ph), n, f"q, call {call + 1}")
        check_reduce(host(s), host(s0), _abs_gemvt(Ah, rh), m, f"s, call {call + 1}")


def test_noalloc_rejects_shapes_beyond_the_scratch(built):
    kf = built
    L = kf.lib()
    big = 1 << 15
    st = L.kf_bicgk_noalloc(big, big, 256, big, 256, 256, 256, 256, None)
    assert st == -2
    assert b"bytes of scratch" in L.kf_last_error()
