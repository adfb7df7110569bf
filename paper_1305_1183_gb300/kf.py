"""Thin ctypes binding of libkf (include/kf.h).

Each function has the name of the C entry point it calls and only marshals
arguments: torch tensors become device pointers and sizes, the stream is the
caller's current CUDA stream.  There is no fallback: if libkf is not built
the first call raises.
"""

from __future__ import annotations

import ctypes
import os

import torch

from . import _build

KF_OK = 0
KF_F32, KF_BF16_ROWSCALE, KF_FP8E4M3_ROWSCALE = 0, 1, 2
(KF_SEQ_BICGK, KF_SEQ_GEMVER, KF_SEQ_GESUMMV, KF_SEQ_ATAX, KF_SEQ_AXPYDOT, KF_SEQ_WAXPBY,
 KF_SEQ_GEMV, KF_SEQ_GEMVT, KF_SEQ_DOT, KF_SEQ_SGEMVT) = range(10)

(KF_ERR_INVALID_ARG, KF_ERR_SHAPE, KF_ERR_DTYPE, KF_ERR_ALIGN, KF_ERR_CYCLE, KF_ERR_UNDEFINED_VAR, KF_ERR_CUDA,
 KF_ERR_NO_MEM, KF_ERR_DEVICE_TIMEOUT, KF_ERR_UNSUPPORTED, KF_ERR_WORKSPACE) = range(-1, -12, -1)

STATUS_NAMES = {
    -1: "KF_ERR_INVALID_ARG", -2: "KF_ERR_SHAPE", -3: "KF_ERR_DTYPE", -4: "KF_ERR_ALIGN",
    -5: "KF_ERR_CYCLE", -6: "KF_ERR_UNDEFINED_VAR", -7: "KF_ERR_CUDA", -8: "KF_ERR_NO_MEM",
    -9: "KF_ERR_DEVICE_TIMEOUT", -10: "KF_ERR_UNSUPPORTED", -11: "KF_ERR_WORKSPACE",
}


class KFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

i64 = ctypes.c_int64
vp = ctypes.c_void_p
f32 = ctypes.c_float
sz = ctypes.c_size_t
ci = ctypes.c_int

_SIGS = {
    "kf_version": ([], ctypes.c_char_p),
    "kf_last_error": ([], ctypes.c_char_p),
    "kf_device_sm_count": ([ctypes.POINTER(ci)], ci),
    "kf_workspace_size": ([ci, i64, i64, ci, ctypes.POINTER(sz)], ci),
    "kf_workspace_init": ([vp, sz, vp], ci),
    "kf_workspace_status": ([vp, vp], ci),
    "kf_bicgk": ([i64, i64, vp, i64, ci, vp, vp, vp, vp, vp, vp, sz, vp], ci),
    "kf_gemver": ([i64, vp, i64, vp, vp, vp, vp, vp, vp, f32, f32, vp, i64, vp, vp, vp, sz, vp], ci),
    "kf_madd": ([i64, i64, vp, i64, vp, i64, vp, i64, vp], ci),
    "kf_gemver_single": ([i64, vp, i64, vp, vp, vp, vp, vp, vp, f32, f32, vp, i64, vp, vp, vp, sz, vp], ci),
    "kf_gemver_q": ([i64, vp, i64, ci, vp, vp, vp, vp, vp, vp, vp, f32, f32, vp, i64, vp, vp, vp, vp, sz, vp], ci),
    "kf_gesummv": ([i64, i64, vp, vp, i64, vp, f32, f32, vp, vp, sz, vp], ci),
    "kf_sgemvt": ([i64, i64, vp, i64, vp, vp, f32, f32, vp, vp, vp, sz, vp], ci),
    "kf_sgemvt_single": ([i64, i64, vp, i64, vp, vp, f32, f32, vp, vp, vp, sz, vp], ci),
    "kf_atax": ([i64, i64, vp, i64, vp, vp, vp, sz, vp], ci),
    "kf_axpydot": ([i64, vp, vp, vp, f32, vp, vp, vp, sz, vp], ci),
    "kf_waxpby": ([i64, f32, vp, f32, vp, vp, vp], ci),
    "kf_gemv": ([i64, i64, vp, i64, ci, vp, f32, vp, f32, vp, vp, vp, sz, vp], ci),
    "kf_gemvt": ([i64, i64, vp, i64, ci, vp, f32, vp, f32, vp, vp, vp, sz, vp], ci),
    "kf_ger": ([i64, i64, vp, i64, f32, vp, vp, vp, i64, vp], ci),
    "kf_axpby": ([i64, f32, vp, f32, vp, vp, vp], ci),
    "kf_scal": ([i64, f32, vp, vp, vp], ci),
    "kf_vadd3": ([i64, vp, vp, vp, vp, vp], ci),
    "kf_dot": ([i64, vp, vp, vp, vp, sz, vp], ci),
    "kf_quantize_rows": ([i64, i64, vp, i64, ci, vp, vp, vp], ci),
    "kf_set_matrix_tuning": ([ci, ci, ci, ci, ci], ci),
    "kf_bicgk_noalloc": ([i64, i64, vp, i64, vp, vp, vp, vp, vp], ci),
    "kf_set_wait_limit_ns": ([ctypes.c_uint64], ci),
    "kf_get_wait_limit_ns": ([ctypes.POINTER(ctypes.c_uint64)], ci),
    "kf_wait_probe": ([ctypes.c_uint64, vp, sz, vp, vp], ci),
    "kf_batched_create": ([ci, vp, ci, ci, ctypes.POINTER(vp)], ci),
    "kf_batched_destroy": ([vp], None),
    "kf_batched_workspace_size": ([vp, ctypes.POINTER(sz)], ci),
    "kf_batched_info": ([vp, ctypes.POINTER(ci), ctypes.POINTER(ctypes.c_double)], ci),
    "kf_batched_upload": ([vp, vp, sz, vp], ci),
    "kf_batched_launch": ([vp, vp, sz, vp], ci),
    "kf_batched_graph_create": ([vp, vp, sz, ctypes.POINTER(vp)], ci),
    "kf_batched_graph_launch": ([vp, vp], ci),
    "kf_batched_graph_destroy": ([vp], None),
    "kf_batched_workspace_bound": ([ci, vp, ci, ctypes.POINTER(sz)], ci),
    "kf_batched_autotune": ([ci, vp, ci, vp, sz, vp, ci, ctypes.POINTER(ci), ctypes.POINTER(ctypes.c_float)], ci),
    "kf_autotune_plan": ([vp, ctypes.POINTER(vp), ci, vp, sz, vp, ci, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)], ci),
    "kf_tune_cache_clear": ([], ci),
    "kf_tune_cache_entries": ([ctypes.POINTER(ci)], ci),
    "kf_tune_cache_save": ([ctypes.c_char_p], ci),
    "kf_tune_cache_load": ([ctypes.c_char_p, ctypes.POINTER(ci)], ci),
    "kf_mlp_param_count": ([ci, ci, ctypes.POINTER(ci)], ci),
    "kf_mlp_workspace_size": ([ci, ci, ci, ctypes.POINTER(sz)], ci),
    "kf_mlp_forward": ([vp, ci, ci, vp, ci, vp, vp], ci),
    "kf_mlp_loss_grad": ([vp, ci, ci, vp, vp, ci, vp, vp, vp, sz, vp], ci),
    "kf_mlp_adam": ([vp, vp, vp, vp, ci, ci, f32, f32, f32, f32, vp], ci),
    "kf_script_create": ([ctypes.POINTER(vp)], ci),
    "kf_script_destroy": ([vp], None),
    "kf_script_vector": ([vp, ctypes.c_char_p, i64, ctypes.POINTER(ci)], ci),
    "kf_script_matrix": ([vp, ctypes.c_char_p, i64, i64, ctypes.POINTER(ci)], ci),
    "kf_script_matrix_ld": ([vp, ctypes.c_char_p, i64, i64, i64, ctypes.POINTER(ci)], ci),
    "kf_script_scalar": ([vp, ctypes.c_char_p, ctypes.POINTER(ci)], ci),
    "kf_script_input": ([vp, ci], ci),
    "kf_script_output": ([vp, ci], ci),
    "kf_script_call": ([vp, ci, ctypes.POINTER(ci), ci, ctypes.POINTER(ci), ci, ctypes.POINTER(ctypes.c_double), ci], ci),
    "kf_script_validate": ([vp], ci),
    "kf_plan_count": ([vp, ci, ctypes.POINTER(ci), ctypes.POINTER(ci)], ci),
    "kf_plan_build": ([vp, ctypes.POINTER(ci * 3), ctypes.POINTER(vp)], ci),
    "kf_plan_destroy": ([vp], None),
    "kf_plan_workspace_size": ([vp, ctypes.POINTER(sz)], ci),
    "kf_plan_kernel_count": ([vp, ctypes.POINTER(ci)], ci),
    "kf_plan_predicted_us": ([vp, ctypes.POINTER(ctypes.c_double)], ci),
    "kf_planner_set_model": ([ctypes.c_double, ctypes.c_double], ci),
    "kf_plan_features": ([vp, vp, ctypes.POINTER(ctypes.c_float), ci, ctypes.POINTER(ci)], ci),
    "kf_plan_describe": ([vp, ctypes.c_char_p, sz, ctypes.POINTER(sz)], ci),
    "kf_plan_enumerate_info": ([vp, ci, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ci), ctypes.POINTER(ci)], ci),
    "kf_plan_execute": ([vp, ctypes.POINTER(vp), ci, vp, sz, vp], ci),
    "kf_plan_time": ([vp, ctypes.POINTER(vp), ci, vp, sz, vp, ci, ctypes.POINTER(ctypes.c_float)], ci),
    "kf_get_matrix_tuning": ([ctypes.POINTER(ci)] * 5, ci),
    "kf_set_autotune": ([ci], ci),
    "kf_get_autotune": ([ctypes.POINTER(ci)], ci),
    "kf_plan_select_workspace_size": ([vp, ci, ctypes.POINTER(sz)], ci),
    "kf_plan_select": ([vp, vp, vp, ctypes.POINTER(vp), ci, vp, sz, vp, ctypes.POINTER(vp), vp], ci),
    "kf_plan_time_all": ([vp, ci, ctypes.POINTER(vp), ci, vp, sz, vp, ci, ctypes.POINTER(ctypes.c_float),
                          ctypes.POINTER(ci)], ci),
    "kf_planner_train_workspace_size": ([ci, ci, ctypes.POINTER(sz)], ci),
    "kf_planner_train": ([ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), ci, ci, vp, vp, vp, vp,
                          sz, vp, vp, ctypes.POINTER(ctypes.c_float), ci, ctypes.POINTER(ci)], ci),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libkf.so (built by ``_build.build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libkf is not built ({path} missing): run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ck(status: int):
    if status != KF_OK:
        raise KFError(status, lib().kf_last_error().decode())


def _p(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _st(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _nb(t):
    return 0 if t is None else t.numel() * t.element_size()


_CODE_DTYPES = {KF_F32: (torch.float32,), KF_BF16_ROWSCALE: (torch.int16, torch.bfloat16),
                KF_FP8E4M3_ROWSCALE: (torch.uint8, torch.int8)}


def _mat(A, fmt=KF_F32, name="A"):
    """A matrix operand: the storage format's element type, unit column
    stride (rows may be strided), on a CUDA device."""
    if A is None:
        return
    if fmt in _CODE_DTYPES and A.dtype not in _CODE_DTYPES[fmt]:
        raise TypeError(f"{name}: dtype {A.dtype} does not hold storage format {fmt}")
    if A.dim() != 2 or (A.shape[1] > 1 and A.stride(1) != 1):
        raise ValueError(f"{name}: a 2-D tensor with unit column stride is required")
    if not A.is_cuda:
        raise ValueError(f"{name}: a CUDA tensor is required")


def _vec(*ts):
    """Vector operands: contiguous float32 CUDA tensors (None passes)."""
    for t in ts:
        if t is None or isinstance(t, int):
            continue
        if t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
            raise TypeError("vector operands must be contiguous float32 CUDA tensors")


# ------------------------------------------------------------------ utilities

def kf_version() -> str:
    return lib().kf_version().decode()


def kf_device_sm_count() -> int:
    v = ci(0)
    _ck(lib().kf_device_sm_count(ctypes.byref(v)))
    return v.value


def kf_workspace_size(seq: int, m: int, n: int, fmt: int = KF_F32) -> int:
    b = sz(0)
    _ck(lib().kf_workspace_size(seq, m, n, fmt, ctypes.byref(b)))
    return b.value


def workspace(seq: int, m: int, n: int, fmt: int = KF_F32, device="cuda") -> torch.Tensor:
    """Zero-filled workspace tensor for ``seq`` (torch owns the memory)."""
    nbytes = max(kf_workspace_size(seq, m, n, fmt), 256)
    return torch.zeros(nbytes, dtype=torch.uint8, device=device)


def kf_workspace_status(ws, stream=None):
    _ck(lib().kf_workspace_status(_p(ws), _st(stream)))


def kf_set_matrix_tuning(warps: int, vec: int, unroll: int, groups: int = 0, stages: int = 4):
    _ck(lib().kf_set_matrix_tuning(warps, vec, unroll, groups, stages))


def kf_get_matrix_tuning():
    v = [ci(0) for _ in range(5)]
    _ck(lib().kf_get_matrix_tuning(*[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


# ------------------------------------------------------------------ sequences

def kf_bicgk(A, p, r, q, s, ws, fmt=KF_F32, row_scale=None, lda=None, n=None, stream=None):
    _mat(A, fmt)
    _vec(p, r, q, s, row_scale)
    m = A.shape[0]
    n = A.shape[1] if n is None else n
    if fmt == KF_F32:
        lda = A.stride(0) if lda is None else lda
    else:
        lda = n if lda is None else lda
    _ck(lib().kf_bicgk(m, n, _p(A), lda, fmt, _p(row_scale), _p(p), _p(r), _p(q), _p(s),
                       _p(ws), _nb(ws), _st(stream)))


def kf_gemver(A, u1, v1, u2, v2, y, z, alpha, beta, B, x, w, ws, stream=None):
    _mat(A)
    _mat(B, name="B")
    _vec(u1, v1, u2, v2, y, z, x, w)
    n = A.shape[0]
    _ck(lib().kf_gemver(n, _p(A), A.stride(0), _p(u1), _p(v1), _p(u2), _p(v2), _p(y), _p(z),
                        alpha, beta, _p(B), B.stride(0), _p(x), _p(w), _p(ws), _nb(ws), _st(stream)))


def kf_gemver_single(A, u1, v1, u2, v2, y, z, alpha, beta, B, x, w, ws, stream=None):
    """GEMVER in one cooperative launch (see include/kf.h)."""
    _mat(A)
    _mat(B, name="B")
    _vec(u1, v1, u2, v2, y, z, x, w)
    n = A.shape[0]
    _ck(lib().kf_gemver_single(n, _p(A), A.stride(0), _p(u1), _p(v1), _p(u2), _p(v2), _p(y), _p(z),
                               alpha, beta, _p(B), B.stride(0), _p(x), _p(w), _p(ws), _nb(ws), _st(stream)))


def kf_gemver_q(QA, fmt, sA, u1, v1, u2, v2, y, z, alpha, beta, QB, sB, x, w, ws, stream=None):
    """GEMVER on row-scaled codes (int16 BF16 or uint8 E4M3 tensors, n x n);
    writes codes QB and scales sB of B, x and w."""
    if fmt != KF_F32:  # KF_F32 codes are the library's to refuse (KF_ERR_DTYPE)
        _mat(QA, fmt, "QA")
        _mat(QB, fmt, "QB")
    _vec(sA, u1, v1, u2, v2, y, z, sB, x, w)
    n = QA.shape[0]
    _ck(lib().kf_gemver_q(n, _p(QA), QA.stride(0), fmt, _p(sA), _p(u1), _p(v1), _p(u2), _p(v2), _p(y), _p(z),
                          alpha, beta, _p(QB), QB.stride(0), _p(sB), _p(x), _p(w), _p(ws), _nb(ws), _st(stream)))


def kf_gesummv(A, B, x, alpha, beta, y, ws, stream=None):
    _mat(A)
    _mat(B, name="B")
    _vec(x, y)
    m, n = A.shape
    assert A.stride(0) == B.stride(0)
    _ck(lib().kf_gesummv(m, n, _p(A), _p(B), A.stride(0), _p(x), alpha, beta, _p(y),
                         _p(ws), _nb(ws), _st(stream)))


def kf_sgemvt(A, y, z, alpha, beta, x, w, ws, stream=None):
    _mat(A)
    _vec(y, z, x, w)
    m, n = A.shape
    _ck(lib().kf_sgemvt(m, n, _p(A), A.stride(0), _p(y), _p(z), alpha, beta, _p(x), _p(w), _p(ws), _nb(ws),
                        _st(stream)))


def kf_sgemvt_single(A, y, z, alpha, beta, x, w, ws, stream=None):
    """SGEMVT in one cooperative launch (see include/kf.h)."""
    _mat(A)
    _vec(y, z, x, w)
    m, n = A.shape
    _ck(lib().kf_sgemvt_single(m, n, _p(A), A.stride(0), _p(y), _p(z), alpha, beta, _p(x), _p(w), _p(ws),
                               _nb(ws), _st(stream)))


def kf_atax(A, x, y, ws, stream=None):
    _mat(A)
    _vec(x, y)
    m, n = A.shape
    _ck(lib().kf_atax(m, n, _p(A), A.stride(0), _p(x), _p(y), _p(ws), _nb(ws), _st(stream)))


def kf_axpydot(w, v, u, alpha, z, r, ws, stream=None):
    _ck(lib().kf_axpydot(w.numel(), _p(w), _p(v), _p(u), alpha, _p(z), _p(r), _p(ws), _nb(ws),
                         _st(stream)))


def kf_waxpby(alpha, x, beta, y, w, stream=None):
    _ck(lib().kf_waxpby(x.numel(), alpha, _p(x), beta, _p(y), _p(w), _st(stream)))


# ------------------------------------------------------------------ elementaries

def kf_gemv(A, x, y, ws, alpha=1.0, beta=0.0, y0=None, fmt=KF_F32, row_scale=None, n=None,
            stream=None):
    _mat(A, fmt)
    _vec(x, y, y0, row_scale)
    m = A.shape[0]
    n = A.shape[1] if n is None else n
    lda = A.stride(0) if fmt == KF_F32 else n
    _ck(lib().kf_gemv(m, n, _p(A), lda, fmt, _p(row_scale), alpha, _p(x), beta, _p(y0), _p(y),
                      _p(ws), _nb(ws), _st(stream)))


def kf_gemvt(A, y, x, ws, alpha=1.0, beta=0.0, x0=None, fmt=KF_F32, row_scale=None, n=None,
             stream=None):
    _mat(A, fmt)
    _vec(y, x, x0, row_scale)
    m = A.shape[0]
    n = A.shape[1] if n is None else n
    lda = A.stride(0) if fmt == KF_F32 else n
    _ck(lib().kf_gemvt(m, n, _p(A), lda, fmt, _p(row_scale), alpha, _p(y), beta, _p(x0), _p(x),
                       _p(ws), _nb(ws), _st(stream)))


def kf_ger(A, u, v, B, alpha=1.0, stream=None):
    _mat(A)
    _mat(B, name="B")
    _vec(u, v)
    m, n = A.shape
    _ck(lib().kf_ger(m, n, _p(A), A.stride(0), alpha, _p(u), _p(v), _p(B), B.stride(0), _st(stream)))


def kf_axpby(alpha, x, beta, y, out, stream=None):
    _ck(lib().kf_axpby(x.numel(), alpha, _p(x), beta, _p(y), _p(out), _st(stream)))


def kf_scal(alpha, x, out, stream=None):
    _ck(lib().kf_scal(x.numel(), alpha, _p(x), _p(out), _st(stream)))


def kf_vadd3(w, y, z, out, stream=None):
    _ck(lib().kf_vadd3(w.numel(), _p(w), _p(y), _p(z), _p(out), _st(stream)))


def kf_madd(A, B, C, stream=None):
    """C = A + B (2-D tensors with unit column stride)."""
    m, n = A.shape
    _ck(lib().kf_madd(m, n, _p(A), A.stride(0), _p(B), B.stride(0), _p(C), C.stride(0), _st(stream)))


def kf_dot(x, y, out, ws, stream=None):
    _ck(lib().kf_dot(x.numel(), _p(x), _p(y), _p(out), _p(ws), _nb(ws), _st(stream)))


def kf_quantize_rows(A, fmt, Q, row_scale, stream=None):
    m, n = A.shape
    _ck(lib().kf_quantize_rows(m, n, _p(A), A.stride(0), fmt, _p(Q), _p(row_scale), _st(stream)))


# ------------------------------------------------------------------ bounded waits

def kf_set_wait_limit_ns(limit_ns: int):
    _ck(lib().kf_set_wait_limit_ns(int(limit_ns)))


def kf_get_wait_limit_ns() -> int:
    v = ctypes.c_uint64(0)
    _ck(lib().kf_get_wait_limit_ns(ctypes.byref(v)))
    return v.value


def kf_wait_probe(limit_ns, ws, waited=None, stream=None):
    """Enqueue a wait that runs out after limit_ns (see include/kf.h)."""
    _ck(lib().kf_wait_probe(int(limit_ns), _p(ws), _nb(ws), _p(waited), _st(stream)))


# ------------------------------------------------------------------ no workspace

KF_BICGK_NOALLOC_SCRATCH_BYTES = 8 << 20


def kf_bicgk_noalloc(A, p, r, q, s, stream=None):
    """BiCGK with the library's fixed device scratch instead of a workspace
    (for callers that cannot allocate); see include/kf.h."""
    _mat(A)
    _vec(p, r, q, s)
    m, n = A.shape
    _ck(lib().kf_bicgk_noalloc(m, n, _p(A), A.stride(0), _p(p), _p(r), _p(q), _p(s), _st(stream)))


# ------------------------------------------------------------------ scripts and plans

KF_OP_AXPBY, KF_OP_SCAL, KF_OP_DOT, KF_OP_VADD, KF_OP_GEMV, KF_OP_GEMVT, KF_OP_GER = range(7)
OPS = {"AXPBY": 0, "SCAL": 1, "DOT": 2, "VADD": 3, "GEMV": 4, "GEMVT": 5, "GER": 6}
KF_PLAN_UNFUSED, KF_PLAN_GREEDY, KF_PLAN_ANALYTIC, KF_PLAN_INDEX = range(4)
KF_SELECT_ANALYTIC, KF_SELECT_MLP, KF_SELECT_EXHAUSTIVE = range(3)
NFEATURES = 16


class _SelectOptions(ctypes.Structure):
    _fields_ = [("mode", ci), ("max_plans", ci), ("top_k", ci), ("reps", ci), ("margin", ctypes.c_float)]


class _CostModel(ctypes.Structure):
    _fields_ = [("params", vp), ("mean", ctypes.c_float * 16), ("inv_std", ctypes.c_float * 16),
                ("analytic_weight", ctypes.c_float)]


class _SelectInfo(ctypes.Structure):
    _fields_ = [("index", ci), ("count", ci), ("timed", ci), ("best_ms", ctypes.c_float),
                ("predicted", ctypes.c_double)]


class CostModel:
    """Learned plan cost model: device parameters of the kf_mlp network
    (16 inputs, 64 hidden units), the host feature standardisation and the
    weight of ln(analytic ms) added to the network's output."""

    def __init__(self, params, mean, inv_std, analytic_weight=0.0):
        self.params = params
        self.mean = [float(x) for x in mean]
        self.inv_std = [float(x) for x in inv_std]
        self.analytic_weight = float(analytic_weight)
        assert len(self.mean) == NFEATURES and len(self.inv_std) == NFEATURES

    def _c(self):
        c = _CostModel()
        c.params = _p(self.params)
        for i in range(NFEATURES):
            c.mean[i] = self.mean[i]
            c.inv_std[i] = self.inv_std[i]
        c.analytic_weight = self.analytic_weight
        return c

    def save(self, path):
        import numpy as np
        np.savez(path, params=self.params.detach().float().cpu().numpy(), mean=np.array(self.mean),
                 inv_std=np.array(self.inv_std), analytic_weight=np.array(self.analytic_weight))

    @staticmethod
    def load(path, device="cuda"):
        import numpy as np
        z = np.load(path)
        return CostModel(torch.tensor(z["params"], dtype=torch.float32, device=device), z["mean"], z["inv_std"],
                         float(z["analytic_weight"]))


class Script:
    """A script of elementary calls (kf_script_* entry points)."""

    def __init__(self):
        h = vp()
        _ck(lib().kf_script_create(ctypes.byref(h)))
        self.h = h
        self.ids = {}
        self.kinds = {}
        self.shapes = {}
        self.lds = {}  # matrix row strides as declared

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.kf_script_destroy(self.h)
            self.h = None

    def vector(self, name, n):
        i = ci(0)
        _ck(lib().kf_script_vector(self.h, name.encode(), n, ctypes.byref(i)))
        self.ids[name] = i.value; self.kinds[name] = "v"; self.shapes[name] = (n,)
        return i.value

    def matrix(self, name, m, n, ld=None):
        """An m x n FP32 matrix; ld: its row stride in elements (default n),
        for a view of a wider array (bind the tensor of the view)."""
        i = ci(0)
        if ld is None:
            _ck(lib().kf_script_matrix(self.h, name.encode(), m, n, ctypes.byref(i)))
        else:
            _ck(lib().kf_script_matrix_ld(self.h, name.encode(), m, n, ld, ctypes.byref(i)))
        self.ids[name] = i.value; self.kinds[name] = "m"; self.shapes[name] = (m, n)
        self.lds[name] = n if ld is None else ld
        return i.value

    def scalar(self, name):
        i = ci(0)
        _ck(lib().kf_script_scalar(self.h, name.encode(), ctypes.byref(i)))
        self.ids[name] = i.value; self.kinds[name] = "s"; self.shapes[name] = (1,)
        return i.value

    def input(self, *names):
        for nm in names:
            _ck(lib().kf_script_input(self.h, self.ids[nm]))

    def output(self, *names):
        for nm in names:
            _ck(lib().kf_script_output(self.h, self.ids[nm]))

    def call(self, op, outs, ins, scalars=()):
        o = (ci * len(outs))(*[self.ids[x] for x in outs])
        i = (ci * len(ins))(*[self.ids[x] for x in ins])
        s = (ctypes.c_double * max(1, len(scalars)))(*scalars)
        _ck(lib().kf_script_call(self.h, OPS[op], o, len(outs), i, len(ins), s, len(scalars)))

    def validate(self):
        _ck(lib().kf_script_validate(self.h))

    def count_plans(self, cap=20000):
        c, t = ci(0), ci(0)
        _ck(lib().kf_plan_count(self.h, cap, ctypes.byref(c), ctypes.byref(t)))
        return c.value, bool(t.value)

    def enumerate_info(self, cap=2000):
        """(features [count x 16], analytic predictions [count], kernel counts [count])."""
        import numpy as np
        f = (ctypes.c_float * (cap * 16))()
        p = (ctypes.c_double * cap)()
        kk = (ci * cap)()
        c = ci(0)
        _ck(lib().kf_plan_enumerate_info(self.h, cap, f, p, kk, ctypes.byref(c)))
        n = c.value
        return (np.frombuffer(f, dtype=np.float32)[:n * 16].reshape(n, 16).copy(),
                np.frombuffer(p, dtype=np.float64)[:n].copy(), np.frombuffer(kk, dtype=np.int32)[:n].copy())

    def _bind(self, bindings):
        arr = (vp * len(self.ids))()
        for name, t in bindings.items():
            arr[self.ids[name]] = _p(t)
        return arr, len(self.ids)

    def select_workspace_size(self, max_plans=0):
        b = sz(0)
        _ck(lib().kf_plan_select_workspace_size(self.h, max_plans, ctypes.byref(b)))
        return b.value

    def select(self, mode, bindings=None, ws=None, model=None, top_k=1, reps=3, max_plans=0, margin=0.0,
               stream=None):
        """kf_plan_select: (Plan, info dict with index, count, timed, best_ms, predicted)."""
        opt = _SelectOptions(mode, max_plans, top_k, reps, margin)
        cm = model._c() if model is not None else None
        arr, nv = self._bind(bindings) if bindings else (None, 0)
        h = vp()
        info = _SelectInfo()
        _ck(lib().kf_plan_select(self.h, ctypes.byref(opt), ctypes.byref(cm) if cm is not None else None, arr, nv,
                                 _p(ws) if ws is not None else None, _nb(ws) if ws is not None else 0,
                                 _st(stream) if mode != KF_SELECT_ANALYTIC else None,
                                 ctypes.byref(h), ctypes.byref(info)))
        return Plan(h, self), {k: getattr(info, k) for k, _ in _SelectInfo._fields_}

    def time_all(self, bindings, ws, reps=3, max_plans=0, stream=None):
        """kf_plan_time_all: median ms of every enumerated plan (numpy array)."""
        import numpy as np
        cap = max_plans if max_plans > 0 else 2000
        ms = (ctypes.c_float * cap)()
        c = ci(0)
        arr, nv = self._bind(bindings)
        _ck(lib().kf_plan_time_all(self.h, max_plans, arr, nv, _p(ws), _nb(ws), _st(stream), reps, ms, ctypes.byref(c)))
        return np.frombuffer(ms, dtype=np.float32)[:c.value].astype(np.float64)

    def plan(self, mode=KF_PLAN_ANALYTIC, index=0, max_plans=0):
        opt = (ci * 3)(mode, max_plans, index)
        h = vp()
        _ck(lib().kf_plan_build(self.h, ctypes.byref(opt), ctypes.byref(h)))
        return Plan(h, self)


class Plan:
    def __init__(self, h, script):
        self.h = h
        self.script = script

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.kf_plan_destroy(self.h)
            self.h = None

    def workspace_size(self):
        b = sz(0)
        _ck(lib().kf_plan_workspace_size(self.h, ctypes.byref(b)))
        return b.value

    def kernel_count(self):
        n = ci(0)
        _ck(lib().kf_plan_kernel_count(self.h, ctypes.byref(n)))
        return n.value

    def predicted_us(self):
        d = ctypes.c_double(0)
        _ck(lib().kf_plan_predicted_us(self.h, ctypes.byref(d)))
        return d.value

    def features(self):
        buf = (ctypes.c_float * 64)()
        n = ci(0)
        _ck(lib().kf_plan_features(self.script.h, self.h, buf, 64, ctypes.byref(n)))
        return list(buf[:n.value])

    def describe(self):
        need = sz(0)
        _ck(lib().kf_plan_describe(self.h, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        _ck(lib().kf_plan_describe(self.h, buf, need.value, ctypes.byref(need)))
        import json
        return json.loads(buf.value.decode())

    def _bind(self, bindings):
        nv = len(self.script.ids)
        arr = (vp * nv)()
        for name, t in bindings.items():
            ld = self.script.lds.get(name)
            if ld is not None and isinstance(t, torch.Tensor) and t.dim() == 2 and t.shape[0] > 1:
                if t.stride(1) != 1 or t.stride(0) != ld:
                    raise ValueError(f"matrix {name}: strides {t.stride()} do not match the declared row stride {ld}")
            arr[self.script.ids[name]] = _p(t)
        return arr, nv

    def execute(self, bindings, ws, stream=None):
        arr, nv = self._bind(bindings)
        _ck(lib().kf_plan_execute(self.h, arr, nv, _p(ws), _nb(ws), _st(stream)))

    def autotune(self, bindings, ws, reps=5, stream=None):
        """Tune every kernel of the plan on the bound data; returns
        (tuned_ms, previous_ms), sums over the kernels of median times."""
        arr, nv = self._bind(bindings)
        a, b = ctypes.c_float(0), ctypes.c_float(0)
        _ck(lib().kf_autotune_plan(self.h, arr, nv, _p(ws), _nb(ws), _st(stream), reps, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def time(self, bindings, ws, reps=5, stream=None):
        arr, nv = self._bind(bindings)
        ms = ctypes.c_float(0)
        _ck(lib().kf_plan_time(self.h, arr, nv, _p(ws), _nb(ws), _st(stream), reps, ctypes.byref(ms)))
        return ms.value


def kf_planner_set_model(bw_gbs, launch_us):
    _ck(lib().kf_planner_set_model(bw_gbs, launch_us))


# ------------------------------------------------------------------ batched


class BatchDesc(ctypes.Structure):
    _fields_ = [("m", i64), ("n", i64), ("lda", i64), ("A", vp), ("B", vp), ("x", vp), ("r", vp),
                ("y", vp), ("s", vp), ("alpha", f32), ("beta", f32)]


def _desc_array(descs):
    arr = (BatchDesc * max(1, len(descs)))()
    for i, d in enumerate(descs):
        arr[i] = BatchDesc(d["m"], d["n"], d.get("lda", d["n"]), _p(d.get("A")), _p(d.get("B")),
                           _p(d.get("x")), _p(d.get("r")), _p(d.get("y")), _p(d.get("s")),
                           d.get("alpha", 1.0), d.get("beta", 0.0))
    return arr


def kf_batched_autotune(seq, descs, reps=5, stream=None):
    """Best tile height for the batch (library-side empirical search)."""
    arr = _desc_array(descs)
    b = sz(0)
    _ck(lib().kf_batched_workspace_bound(seq, ctypes.cast(arr, vp), len(descs), ctypes.byref(b)))
    ws = torch.zeros(max(b.value, 256), dtype=torch.uint8, device="cuda")
    best, ms = ci(0), ctypes.c_float(0)
    _ck(lib().kf_batched_autotune(seq, ctypes.cast(arr, vp), len(descs), _p(ws), _nb(ws), _st(stream), reps,
                                  ctypes.byref(best), ctypes.byref(ms)))
    return best.value, ms.value


class Batched:
    """kf_batched_* handle: `descs` is a list of dicts with m, n, lda and
    device pointers A, B, x, r, y, s (ints or tensors), alpha, beta."""

    def __init__(self, seq, descs, band_rows=0):
        arr = _desc_array(descs)
        h = vp()
        _ck(lib().kf_batched_create(seq, ctypes.cast(arr, vp), len(descs), band_rows, ctypes.byref(h)))
        self.h = h
        self.graph = None

    def __del__(self):
        if getattr(self, "graph", None) and _lib is not None:
            _lib.kf_batched_graph_destroy(self.graph)
        if getattr(self, "h", None) and _lib is not None:
            _lib.kf_batched_destroy(self.h)

    def workspace_size(self):
        b = sz(0)
        _ck(lib().kf_batched_workspace_size(self.h, ctypes.byref(b)))
        return b.value

    def info(self):
        t, b = ci(0), ctypes.c_double(0)
        _ck(lib().kf_batched_info(self.h, ctypes.byref(t), ctypes.byref(b)))
        return t.value, b.value

    def upload(self, ws, stream=None):
        _ck(lib().kf_batched_upload(self.h, _p(ws), _nb(ws), _st(stream)))

    def launch(self, ws, stream=None):
        _ck(lib().kf_batched_launch(self.h, _p(ws), _nb(ws), _st(stream)))

    def capture(self, ws):
        g = vp()
        _ck(lib().kf_batched_graph_create(self.h, _p(ws), _nb(ws), ctypes.byref(g)))
        self.graph = g
        return g

    def replay(self, stream=None):
        _ck(lib().kf_batched_graph_launch(self.graph, _st(stream)))


def kf_set_autotune(reps):
    """Tuning on first use: reps > 0 searches every new tuning key on its first launch."""
    _ck(lib().kf_set_autotune(reps))


def kf_get_autotune():
    r = ci(0)
    _ck(lib().kf_get_autotune(ctypes.byref(r)))
    return r.value


def kf_tune_cache_clear():
    _ck(lib().kf_tune_cache_clear())


def kf_tune_cache_entries():
    n = ci(0)
    _ck(lib().kf_tune_cache_entries(ctypes.byref(n)))
    return n.value


def kf_tune_cache_save(path):
    _ck(lib().kf_tune_cache_save(str(path).encode()))


def kf_tune_cache_load(path):
    n = ci(0)
    _ck(lib().kf_tune_cache_load(str(path).encode(), ctypes.byref(n)))
    return n.value


# ------------------------------------------------------------------ cost model

MLP_HIDDEN = 64


def kf_mlp_param_count(d_in, hidden=MLP_HIDDEN):
    c = ci(0)
    _ck(lib().kf_mlp_param_count(d_in, hidden, ctypes.byref(c)))
    return c.value


def kf_mlp_workspace_size(d_in, batch, hidden=MLP_HIDDEN):
    b = sz(0)
    _ck(lib().kf_mlp_workspace_size(d_in, hidden, batch, ctypes.byref(b)))
    return b.value


def kf_mlp_forward(params, X, out, hidden=MLP_HIDDEN, stream=None):
    _ck(lib().kf_mlp_forward(_p(params), X.shape[1], hidden, _p(X), X.shape[0], _p(out), _st(stream)))


def kf_mlp_loss_grad(params, X, y, grad, loss, ws, hidden=MLP_HIDDEN, stream=None):
    _ck(lib().kf_mlp_loss_grad(_p(params), X.shape[1], hidden, _p(X), _p(y), X.shape[0], _p(grad), _p(loss),
                               _p(ws), _nb(ws), _st(stream)))


class _TrainOptions(ctypes.Structure):
    _fields_ = [("epochs", ci), ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("analytic_weight", ctypes.c_float), ("centre_per_script", ci),
                ("loss_every", ci), ("seed", ctypes.c_uint64)]


def kf_planner_train_workspace_size(count, d_in=NFEATURES):
    b = sz(0)
    _ck(lib().kf_planner_train_workspace_size(count, d_in, ctypes.byref(b)))
    return b.value


def kf_planner_train(X, ms, analytic_us, script_ids=None, epochs=3000, lr=3e-3, b1=0.9, b2=0.999, eps=1e-8,
                     analytic_weight=1.0, centre=True, loss_every=500, seed=0, params_init=None, device="cuda",
                     stream=None):
    """Train the plan cost model in the library (kf_planner_train): host
    arrays in, a CostModel (device parameters, standardisation) and the
    recorded losses [(step, loss)] out."""
    import numpy as np
    X = np.ascontiguousarray(X, dtype=np.float32)
    count, d = X.shape
    msd = np.ascontiguousarray(ms, dtype=np.float64)
    pud = np.ascontiguousarray(analytic_us, dtype=np.float64)
    sid = None if script_ids is None else np.ascontiguousarray(script_ids, dtype=np.int64)
    params = torch.empty(kf_mlp_param_count(d), dtype=torch.float32, device=device)
    ws = torch.empty(kf_planner_train_workspace_size(count, d), dtype=torch.uint8, device=device)
    opt = _TrainOptions(epochs, lr, b1, b2, eps, analytic_weight, 1 if centre else 0, loss_every, seed)
    cap = epochs // loss_every + 2 if loss_every > 0 else 2
    losses = (ctypes.c_float * cap)()
    nl = ci(0)
    cm = _CostModel()
    fp, dp = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)
    _ck(lib().kf_planner_train(X.ctypes.data_as(fp), msd.ctypes.data_as(dp), pud.ctypes.data_as(dp),
                               None if sid is None else sid.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               count, d, ctypes.byref(opt), _p(params_init), _p(params), _p(ws), _nb(ws),
                               _st(stream), ctypes.byref(cm), losses, cap, ctypes.byref(nl)))
    steps = [1] + ([t for t in range(loss_every, epochs + 1, loss_every)] if loss_every > 0 else []) + [epochs + 1]
    hist = list(zip(steps, [float(losses[i]) for i in range(min(nl.value, cap))]))
    model = CostModel(params, list(cm.mean), list(cm.inv_std), cm.analytic_weight)
    return model, hist


def kf_mlp_adam(params, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    _ck(lib().kf_mlp_adam(_p(params), _p(grad), _p(m), _p(v), params.numel(), step, lr, b1, b2, eps, _st(stream)))
