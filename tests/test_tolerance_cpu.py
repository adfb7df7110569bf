"""The acceptance checks used by every parity test accept and reject at the
stated bound (no GPU): relative error 1e-5 sqrt(n), normwise and
componentwise against the sum of |terms|; 4 FP32 ulps of the sum of |terms|
for map-only results."""

import numpy as np
import pytest

from tolerance import EPS32, check_map, check_reduce, rel_tol


def test_rel_tol_values():
    assert rel_tol(1) == 1e-5 and rel_tol(0) == 1e-5
    assert rel_tol(16384) == pytest.approx(1.28e-3)
    assert rel_tol(1 << 26) == pytest.approx(1e-5 * 8192)


def test_normwise_bound():
    n = 10000                                   # tol 1e-3
    ref = np.array([1.0, -2.0, 0.5])
    scale = np.full(3, 1e9)                     # componentwise check out of the way
    check_reduce(ref + np.array([0.0, 1.99e-3, 0.0]), ref, scale, n)
    with pytest.raises(AssertionError, match="normwise"):
        check_reduce(ref + np.array([0.0, 2.01e-3, 0.0]), ref, scale, n)


def test_componentwise_bound_guards_cancellation():
    """A small result from large cancelling terms may carry an error up to
    tol times its sum of |terms|, not more, even when normwise passes."""
    n = 100                                     # tol 1e-4
    ref = np.array([1000.0, 1e-3])
    scale = np.array([1000.0, 50.0])            # the second result cancels terms summing to 50
    check_reduce(ref + np.array([0.0, 4.9e-3]), ref, scale, n)
    with pytest.raises(AssertionError, match="componentwise"):
        check_reduce(ref + np.array([0.0, 5.1e-3]), ref, scale, n)


def test_non_finite_and_shape_are_rejected():
    with pytest.raises(AssertionError, match="non-finite"):
        check_reduce(np.array([np.nan, 1.0]), np.array([0.0, 1.0]), np.ones(2), 4)
    with pytest.raises(AssertionError):
        check_reduce(np.ones(3), np.ones(2), np.ones(2), 4)


def test_map_bound_is_four_ulps_of_the_terms():
    ref = np.array([1.0, 3.0])
    scale = np.array([2.0, 6.0])
    check_map(ref + 3.9 * EPS32 * scale, ref, scale)
    with pytest.raises(AssertionError, match="map check"):
        check_map(ref + 4.1 * EPS32 * scale, ref, scale)
