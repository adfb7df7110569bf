"""Acceptance checks for FP32 results against the FP64 oracle.

Tolerance: relative error 1e-5 * sqrt(n), n the reduction length of the
result (for chained results, the longer stage).  Two checks both hold:
  normwise      max|yhat - y| / max|y|           <= 1e-5 sqrt(n)
  componentwise |yhat_i - y_i| <= 1e-5 sqrt(n) * scale_i
where scale_i is the sum of |terms| of result i (|A||x| for a matrix-vector
product), the usual backward-error scale of a dot product, which keeps the
check meaningful where cancellation makes y_i small.
Map-only results (no reduction) must be within 4 ulp-of-FP32 of the sum of
|terms|: |e_hat - e| <= 4 * 2**-24 * scale.
"""

import numpy as np

EPS32 = 2.0 ** -24


def rel_tol(n: int) -> float:
    return 1e-5 * np.sqrt(max(int(n), 1))


def check_reduce(got, ref, scale, n, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.asarray(scale, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    tol = rel_tol(n)
    err = np.abs(got - ref)
    denom = max(np.max(np.abs(ref)), 1e-300)
    nw = np.max(err) / denom if err.size else 0.0
    assert nw <= tol, f"{what}: normwise rel err {nw:.3e} > {tol:.3e}"
    bad = err > tol * scale + 1e-300
    assert not np.any(bad), (
        f"{what}: componentwise check fails at {np.flatnonzero(bad)[:8]} "
        f"err={err[bad][:4]} bound={(tol * scale)[bad][:4]}")
    return nw


def check_map(got, ref, scale, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(got - ref)
    bound = 4 * EPS32 * np.asarray(scale, dtype=np.float64)
    bad = err > bound
    assert not np.any(bad), f"{what}: map check fails, max err {err.max():.3e}"
