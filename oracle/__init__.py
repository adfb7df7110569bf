"""FP64 CPU oracle for the fused BLAS sequences.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package.  It shares no code
with the CUDA path and never imports it.

The arithmetic lives in ``kf_oracle.c`` (plain double loops, one function per
definition in the paper's Table 1) and in ``mlp.py`` / ``script.py``.  This
file builds the C part with gcc and wraps it with ctypes + numpy.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libkf_oracle.so")
_SRC = os.path.join(_HERE, "kf_oracle.c")

_lib = None


SOURCE = _SRC


def compile_source(src: str, out: str) -> str:
    """Compile one oracle C source into a shared library (gcc, -O2, strict IEEE)."""
    subprocess.run(
        ["gcc", "-O2", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
         "-std=c11", "-o", out, src, "-lm"],
        check=True,
    )
    return out


def build(force: bool = False) -> str:
    """Compile kf_oracle.c into the package's shared library when it is stale."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        compile_source(_SRC, tmp)
        os.replace(tmp, _SO)
    return _SO


def lib():
    """The loaded oracle library (built on first use)."""
    global _lib
    if _lib is None:
        build()
        _lib = load(_SO)
    return _lib


def load(path: str):
    """Load a compiled oracle library from ``path`` and declare its signatures."""
    L = ctypes.CDLL(path)
    d = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    dbl = ctypes.c_double
    vp = ctypes.c_void_p
    fp = ctypes.POINTER(ctypes.c_float)
    L.kfo_gemv.argtypes = [i64, i64, d, i64, d, dbl, dbl, d, d]
    L.kfo_gemvt.argtypes = [i64, i64, d, i64, d, dbl, dbl, d, d]
    L.kfo_ger.argtypes = [i64, i64, d, i64, dbl, d, d, d, i64]
    L.kfo_madd.argtypes = [i64, i64, d, d, d]
    L.kfo_axpby.argtypes = [i64, dbl, d, dbl, d, d]
    L.kfo_vadd3.argtypes = [i64, d, d, d, d]
    L.kfo_dot.argtypes = [i64, d, d]
    L.kfo_dot.restype = dbl
    L.kfo_bicgk.argtypes = [i64, i64, d, i64, d, d, d, d]
    L.kfo_gemver.argtypes = [i64, d, i64, d, d, d, d, d, d, dbl, dbl, d, d, d]
    L.kfo_gesummv.argtypes = [i64, i64, d, d, i64, d, dbl, dbl, d]
    L.kfo_atax.argtypes = [i64, i64, d, i64, d, d, d]
    L.kfo_axpydot.argtypes = [i64, d, d, d, dbl, d]
    L.kfo_axpydot.restype = dbl
    L.kfo_waxpby.argtypes = [i64, dbl, d, dbl, d, d]
    L.kfo_abs_gemv.argtypes = [i64, i64, d, i64, d, d]
    L.kfo_abs_gemvt.argtypes = [i64, i64, d, i64, d, d]
    L.kfo_quantize_rows.argtypes = [i64, i64, fp, i64, ctypes.c_int, vp, fp]
    L.kfo_dequantize_rows.argtypes = [i64, i64, vp, ctypes.c_int, fp, d]
    L.kfo_gemver_rowscaled_store.argtypes = [i64, vp, ctypes.c_int, fp, fp, fp, fp, fp, vp, fp]
    L.kfo_bf16_value.argtypes = [ctypes.c_uint16]
    L.kfo_bf16_value.restype = dbl
    L.kfo_e4m3_value.argtypes = [ctypes.c_uint8]
    L.kfo_e4m3_value.restype = dbl
    L.kfo_bf16_code.argtypes = [ctypes.c_float]
    L.kfo_bf16_code.restype = ctypes.c_uint16
    L.kfo_e4m3_code.argtypes = [ctypes.c_float]
    L.kfo_e4m3_code.restype = ctypes.c_uint8
    return L


def _d(a) -> np.ndarray:
    """Exact widening of FP32 (or already FP64) inputs to a contiguous double array."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------- elementaries

def gemv(A, x, alpha=1.0, beta=0.0, y0=None):
    A = _d(A); x = _d(x)
    m, n = A.shape
    y = np.empty(m)
    y0d = _d(y0) if y0 is not None else np.zeros(m)
    lib().kfo_gemv(m, n, _p(A), n, _p(x), alpha, beta, _p(y0d), _p(y))
    return y


def gemvt(A, y, alpha=1.0, beta=0.0, x0=None):
    A = _d(A); y = _d(y)
    m, n = A.shape
    x = np.empty(n)
    x0d = _d(x0) if x0 is not None else np.zeros(n)
    lib().kfo_gemvt(m, n, _p(A), n, _p(y), alpha, beta, _p(x0d), _p(x))
    return x


def ger(A, u, v, alpha=1.0):
    A = _d(A); u = _d(u); v = _d(v)
    m, n = A.shape
    B = np.empty((m, n))
    lib().kfo_ger(m, n, _p(A), n, alpha, _p(u), _p(v), _p(B), n)
    return B


def madd(A, B):
    A = _d(A); B = _d(B)
    C = np.empty_like(A)
    lib().kfo_madd(A.shape[0], A.shape[1], _p(A), _p(B), _p(C))
    return C


def axpby(alpha, x, beta, y):
    x = _d(x); y = _d(y)
    out = np.empty(x.shape[0])
    lib().kfo_axpby(x.shape[0], alpha, _p(x), beta, _p(y), _p(out))
    return out


def vadd3(w, y, z):
    w = _d(w); y = _d(y); z = _d(z)
    out = np.empty(w.shape[0])
    lib().kfo_vadd3(w.shape[0], _p(w), _p(y), _p(z), _p(out))
    return out


def dot(x, y):
    x = _d(x); y = _d(y)
    return lib().kfo_dot(x.shape[0], _p(x), _p(y))


# ---------------------------------------------------------------- sequences

def bicgk(A, p, r):
    """Returns (q, s) = (A p, A^T r)."""
    A = _d(A); p = _d(p); r = _d(r)
    m, n = A.shape
    q = np.empty(m); s = np.empty(n)
    lib().kfo_bicgk(m, n, _p(A), n, _p(p), _p(r), _p(q), _p(s))
    return q, s


def gemver(A, u1, v1, u2, v2, y, z, alpha, beta):
    """Returns (B, x, w)."""
    A = _d(A)
    n = A.shape[0]
    args = [_d(a) for a in (u1, v1, u2, v2, y, z)]
    B = np.empty((n, n)); x = np.empty(n); w = np.empty(n)
    lib().kfo_gemver(n, _p(A), n, *[_p(a) for a in args], alpha, beta, _p(B), _p(x), _p(w))
    return B, x, w


def gesummv(A, B, x, alpha, beta):
    A = _d(A); B = _d(B); x = _d(x)
    m, n = A.shape
    y = np.empty(m)
    lib().kfo_gesummv(m, n, _p(A), _p(B), n, _p(x), alpha, beta, _p(y))
    return y


def sgemvt(A, y, z, alpha, beta):
    """SGEMVT of Table 1: returns (x, w) with x = beta A^T y + z and
    w = alpha A x (the FP64 x), the script's calls in order."""
    x = gemvt(A, y, alpha=beta, beta=1.0, x0=z)
    w = gemv(A, x, alpha=alpha)
    return x, w


def atax(A, x):
    """Returns (y, t) with t = A x and y = A^T t."""
    A = _d(A); x = _d(x)
    m, n = A.shape
    t = np.empty(m); y = np.empty(n)
    lib().kfo_atax(m, n, _p(A), n, _p(x), _p(t), _p(y))
    return y, t


def axpydot(w, v, u, alpha):
    """Returns (z, r)."""
    w = _d(w); v = _d(v); u = _d(u)
    z = np.empty(w.shape[0])
    r = lib().kfo_axpydot(w.shape[0], _p(w), _p(v), _p(u), alpha, _p(z))
    return z, r


def waxpby(alpha, x, beta, y):
    x = _d(x); y = _d(y)
    w = np.empty(x.shape[0])
    lib().kfo_waxpby(x.shape[0], alpha, _p(x), beta, _p(y), _p(w))
    return w


def abs_gemv(A, x):
    A = _d(A); x = _d(x)
    m, n = A.shape
    out = np.empty(m)
    lib().kfo_abs_gemv(m, n, _p(A), n, _p(x), _p(out))
    return out


def abs_gemvt(A, y):
    A = _d(A); y = _d(y)
    m, n = A.shape
    out = np.empty(n)
    lib().kfo_abs_gemvt(m, n, _p(A), n, _p(y), _p(out))
    return out


# ---------------------------------------------------------------- low precision

FMT_BF16 = 1
FMT_E4M3 = 2


def quantize_rows(A, fmt):
    """Row-scaled quantisation of an FP32 matrix.  Returns (codes, scale):
    codes uint16 (BF16 bit patterns) or uint8 (E4M3 bit patterns), scale float32."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float32))
    m, n = A.shape
    codes = np.empty((m, n), dtype=np.uint8 if fmt == FMT_E4M3 else np.uint16)
    scale = np.empty(m, dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    lib().kfo_quantize_rows(m, n, A.ctypes.data_as(fp), n, fmt,
                            codes.ctypes.data_as(ctypes.c_void_p), scale.ctypes.data_as(fp))
    return codes, scale


def dequantize_rows(codes, scale, fmt):
    codes = np.ascontiguousarray(codes)
    scale = np.ascontiguousarray(np.asarray(scale, dtype=np.float32))
    m, n = codes.shape
    out = np.empty((m, n))
    fp = ctypes.POINTER(ctypes.c_float)
    lib().kfo_dequantize_rows(m, n, codes.ctypes.data_as(ctypes.c_void_p), fmt,
                              scale.ctypes.data_as(fp), _p(out))
    return out


def gemver_rowscaled(QA, sA, fmt, u1, v1, u2, v2, y, z, alpha, beta):
    """GEMVER on row-scaled codes: returns (QB, sB, Bhat, x, w) with the
    storage rule of kfo_gemver_rowscaled_store, then x = beta Bhat^T y + z and
    w = alpha Bhat x in double on the stored matrix Bhat_ij = sB_i QB_ij."""
    QA = np.ascontiguousarray(QA)
    n = QA.shape[0]
    f32 = [np.ascontiguousarray(np.asarray(a, dtype=np.float32)) for a in (sA, u1, v1, u2, v2)]
    QB = np.empty_like(QA)
    sB = np.empty(n, dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    lib().kfo_gemver_rowscaled_store(n, QA.ctypes.data_as(ctypes.c_void_p), fmt,
                                     *[a.ctypes.data_as(fp) for a in f32],
                                     QB.ctypes.data_as(ctypes.c_void_p), sB.ctypes.data_as(fp))
    Bhat = dequantize_rows(QB, sB, fmt)
    x = gemvt(Bhat, y, alpha=beta, beta=1.0, x0=z)
    w = gemv(Bhat, x, alpha=alpha)
    return QB, sB, Bhat, x, w


def bf16_value(code: int) -> float:
    return lib().kfo_bf16_value(code)


def e4m3_value(code: int) -> float:
    return lib().kfo_e4m3_value(code)


def bf16_code(f: float) -> int:
    return lib().kfo_bf16_code(f)


def e4m3_code(f: float) -> int:
    return lib().kfo_e4m3_code(f)
