"""Bounded device waits: a wait that runs out is reported and the context
stays usable.

Every wait of the library's kernels on data (bulk-copy rings of the staged
matrix pass and of ATAX) gives up after a limit, records the timeout in the
workspace's error word and returns.  kf_wait_probe makes such a wait run out
on purpose, without a fault: it waits on an mbarrier phase that nothing
completes, bounded by a limit of a few microseconds.  The tests check that
the kernel returns, that kf_workspace_status reports KF_ERR_DEVICE_TIMEOUT
once (it clears the word), and that a normal BiCGK afterwards still matches
the FP64 oracle.  A limit set with kf_set_wait_limit_ns well above a copy's
latency leaves the staged kernels' results correct.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import built, dev, host  # noqa: F401
from tolerance import check_reduce

pytestmark = pytest.mark.gpu


def _bicgk_vs_oracle(kf, m, n, seed, ws=None):
    A = synth.uniform((m, n), seed, synth.TID["A"], device=dev())
    p = synth.uniform((n,), seed, synth.TID["p"], device=dev())
    r = synth.uniform((m,), seed, synth.TID["r"], device=dev())
    q, s = torch.empty(m, device=dev()), torch.empty(n, device=dev())
    ws = kf.workspace(kf.KF_SEQ_BICGK, m, n) if ws is None else ws
    kf.kf_bicgk(A, p, r, q, s, ws)
    kf.kf_workspace_status(ws)  # no wait ran out
    Ah, ph, rh = host(A), host(p), host(r)
    qo, so = oracle.bicgk(Ah, ph, rh)
    check_reduce(host(q), qo, np.abs(Ah) @ np.abs(ph), n, "q")
    check_reduce(host(s), so, np.abs(Ah).T @ np.abs(rh), m, "s")


@pytest.mark.parametrize("limit_ns", [5_000, 200_000])
def test_wait_that_runs_out_is_reported(built, limit_ns):
    kf = built
    ws = torch.zeros(256, dtype=torch.uint8, device=dev())
    waited = torch.zeros(1, dtype=torch.int64, device=dev())
    kf.kf_wait_probe(limit_ns, ws, waited)
    torch.cuda.synchronize()  # the kernel returned
    with pytest.raises(kf.KFError) as e:
        kf.kf_workspace_status(ws)
    assert e.value.status == kf.KF_ERR_DEVICE_TIMEOUT
    w = int(waited.item())
    assert limit_ns <= w < 100_000_000, w  # it waited the limit, and no longer than a bounded moment
    kf.kf_workspace_status(ws)  # the status read cleared the word
    # the context is still usable: a normal call matches the oracle
    _bicgk_vs_oracle(kf, 1500, 1300, 51)


def test_staged_kernels_with_a_shorter_limit(built):
    """A limit of 50 ms (far above a copy's latency) on the staged matrix
    pass and on ATAX: no wait runs out and the results match the oracle."""
    kf = built
    old = kf.kf_get_wait_limit_ns()
    assert old == 1_000_000_000
    kf.kf_set_wait_limit_ns(50_000_000)
    kf.kf_set_matrix_tuning(8, 1, 4, 0, 3)
    try:
        assert kf.kf_get_wait_limit_ns() == 50_000_000
        _bicgk_vs_oracle(kf, 3000, 2048, 52)
        m, n = 2000, 1024
        A = synth.uniform((m, n), 53, synth.TID["A"], device=dev())
        x = synth.uniform((n,), 53, synth.TID["x"], device=dev())
        y = torch.empty(n, device=dev())
        ws = kf.workspace(kf.KF_SEQ_ATAX, m, n)
        kf.kf_atax(A, x, y, ws)
        kf.kf_workspace_status(ws)
        Ah, xh = host(A), host(x)
        check_reduce(host(y), oracle.atax(Ah, xh)[0], np.abs(Ah).T @ (np.abs(Ah) @ np.abs(xh)), max(m, n), "y")
    finally:
        kf.kf_set_matrix_tuning(0, 0, 0, 0, 0)
        kf.kf_set_wait_limit_ns(old)
