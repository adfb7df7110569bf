"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the fused-BLAS method: it only turns
(seed, tensor id, element index) into numbers.  Both sides of every parity
check draw their inputs from here, so the oracle and the CUDA path see the
same FP32 values.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-style.  For tensor ``tid`` of
run ``seed`` the 64-bit key is ``mix(mix(seed) + tid)``; element ``i`` is
``mix(key + (i + 1) * GAMMA)``, where ``mix`` is the SplitMix64 output
function (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31) and
GAMMA = 0x9E3779B97F4A7C15.  The top 24 bits ``b`` give the uniform value
``b * 2**-23 - 1`` on a 2**-23 grid in [-1, 1), exact in FP32.

The paper (Section 4.1) states no input values or sizes; the distributions
used here (uniform [-1, 1) for every matrix and vector entry, sizes of the
experiment configurations) are the workload recipe of this project.

Everything is written with torch int64 tensors so the same code runs on the
CPU and on a CUDA device; int64 multiply wraps modulo 2**64 and logical right
shifts are done with a mask.
"""

from __future__ import annotations

import math

import torch

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# Fixed tensor ids per role, so every consumer draws the same values.
TID = {
    "A": 1, "B": 2, "p": 3, "x": 3, "r": 4, "y": 4, "u1": 5, "v1": 6,
    "u2": 7, "v2": 8, "z": 9, "w": 10, "v": 11, "u": 12, "sizes": 13,
    "script": 14, "mlp": 15,
}


def _s64(c: int) -> int:
    """Unsigned 64-bit constant -> the int64 value with the same bits."""
    c &= MASK64
    return c - (1 << 64) if c >= (1 << 63) else c


def _srl(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix_t(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _srl(z, 30)) * _s64(M1)
    z = (z ^ _srl(z, 27)) * _s64(M2)
    return z ^ _srl(z, 31)


def _mix_int(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def key(seed: int, tid: int) -> int:
    return _mix_int(_mix_int(seed) + tid)


def bits(seed: int, tid: int, idx: torch.Tensor) -> torch.Tensor:
    """Raw 64-bit outputs (as int64 bit patterns) for element indices ``idx``."""
    k = _s64(key(seed, tid))
    z = k + (idx.to(torch.int64) + 1) * _s64(GAMMA)
    return _mix_t(z)


def uniform_at(seed: int, tid: int, idx: torch.Tensor) -> torch.Tensor:
    """Uniform [-1, 1) FP32 values on a 2**-23 grid at element indices ``idx``."""
    b = _srl(bits(seed, tid, idx), 40)
    return b.to(torch.float32) * (2.0 ** -23) - 1.0


def integers_at(seed: int, tid: int, idx: torch.Tensor, lo: int = -2, hi: int = 2) -> torch.Tensor:
    """Integer-valued FP32 in [lo, hi] (used for order-independent exact sums)."""
    b = _srl(bits(seed, tid, idx), 40)
    return (b % (hi - lo + 1) + lo).to(torch.float32)


def uniform(shape, seed: int, tid: int, device="cpu") -> torch.Tensor:
    n = math.prod(shape) if len(shape) else 1
    idx = torch.arange(n, dtype=torch.int64, device=device)
    return uniform_at(seed, tid, idx).reshape(shape)


def integers(shape, seed: int, tid: int, lo: int = -2, hi: int = 2, device="cpu") -> torch.Tensor:
    n = math.prod(shape) if len(shape) else 1
    idx = torch.arange(n, dtype=torch.int64, device=device)
    return integers_at(seed, tid, idx, lo, hi).reshape(shape)


def matrix_rows(m: int, n: int, rows, seed: int, tid: int, device="cpu") -> torch.Tensor:
    """Rows ``rows`` of the m x n row-major uniform matrix (tensor ``tid``)."""
    rows = torch.as_tensor(rows, dtype=torch.int64, device=device)
    idx = rows[:, None] * n + torch.arange(n, dtype=torch.int64, device=device)[None, :]
    return uniform_at(seed, tid, idx)


def matrix_cols(m: int, n: int, cols, seed: int, tid: int, device="cpu") -> torch.Tensor:
    """Columns ``cols`` of the m x n row-major uniform matrix, as a (len(cols), m) array."""
    cols = torch.as_tensor(cols, dtype=torch.int64, device=device)
    idx = torch.arange(m, dtype=torch.int64, device=device)[None, :] * n + cols[:, None]
    return uniform_at(seed, tid, idx)


def uniform_scalar(seed: int, tid: int, index: int) -> float:
    """One uniform [-1, 1) value (used for per-call scalars of random scripts)."""
    return float(uniform_at(seed, tid, torch.tensor([index]))[0])


def log_uniform_int(lo: int, hi: int, seed: int, tid: int, count: int, device="cpu") -> torch.Tensor:
    """Sizes round(exp(U * ln(hi/lo) + ln lo)) with U uniform in [0, 1)."""
    idx = torch.arange(count, dtype=torch.int64, device=device)
    u = _srl(bits(seed, tid, idx), 11).to(torch.float64) * (2.0 ** -53)
    v = torch.exp(u * math.log(hi / lo) + math.log(lo))
    return torch.clamp(torch.round(v), lo, hi).to(torch.int64)
