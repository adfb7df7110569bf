"""Benchmark of the fused BLAS-1/BLAS-2 sequence suite on one or more GPUs.

One step = one pass of every fused sequence of the at-scale FP32 suite:
BiCGK 16384 x 16384, GEMVER n = 8192, GESUMMV n = 8192, ATAX 8192 x 8192,
AXPYDOT and WAXPBY n = 2^26 (alpha = 1.5, beta = 1.2, entries uniform in
[-1, 1) from the seeded generator).  Every input is larger than the 129 MB L2
or a vector that a fused kernel keeps on chip, so each step streams from HBM.

Reported value: algorithmic bytes of the suite (bytes each sequence must move
at least once: matrices read/written once, vectors once) / device time, in
GB/s.  Beside it: per-sequence GB/s and fraction of the measured HBM copy
bandwidth, the unfused per-call kernel chain on the same GPU and its speedup,
the same sequences as cuBLAS call chains (context: the paper's comparison
system), the dominant kernel's roofline (against the measured copy, and
against a read-only probe of the library's own dot product), an end-to-end
number through host buffers, the row-scaled BF16 / E4M3 forms, the batched form, and the FP64
CPU oracle's throughput on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU runs (torchrun) are independent replicas: the suite does not shard
into an exchange; every rank runs its own copy and the value is the sum of
bytes over ranks divided by the slowest rank's time.
"""

from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

ALPHA, BETA = 1.5, 1.2
METRIC = "fused-sequence HBM GB/s, % of GB300 peak, speedup vs unfused chain"
WORKLOAD = ("FP32 sequence suite at scale: GEMVER n=8192, GESUMMV n=8192, ATAX 8192x8192, "
            "BiCGK 16384x16384, AXPYDOT and WAXPBY n=2^26; entries uniform[-1,1), seed 0")
NOMINAL_HBM_GBS = 8000.0
FALLBACK_HBM_GBS = 6800.0

FULL = dict(bicgk=(16384, 16384), gemver=8192, gesummv=8192, atax=(8192, 8192), axpydot=1 << 26,
            waxpby=1 << 26)
SMALL = dict(bicgk=(2048, 2048), gemver=1024, gesummv=1024, atax=(1024, 1024), axpydot=1 << 20,
             waxpby=1 << 20)


# ---------------------------------------------------------------- byte model

def algorithmic_bytes(seq: str, size) -> int:
    """Bytes the sequence must move at least once (FP32), per the counting of
    the paper's Section 4.2: only data really transferred to or from memory."""
    f = 4
    if seq == "bicgk":
        m, n = size
        return f * (m * n + 2 * (m + n))             # A; p, r in; q, s out
    if seq == "gemver":
        n = size
        return f * (3 * n * n + 9 * n)               # A read, B written, B read; 9 vectors
    if seq == "gesummv":
        n = size
        return f * (2 * n * n + 2 * n)               # A, B read; x in; y out
    if seq == "atax":
        m, n = size
        return f * (m * n + 2 * n)                   # A read once; x in; y out
    if seq == "axpydot":
        return f * (4 * size + 1)                    # w, v, u in; z, r out
    if seq == "waxpby":
        return f * 3 * size                          # x, y in; w out
    raise KeyError(seq)


def unfused_bytes(seq: str, size) -> int:
    """Bytes of the one-kernel-per-call chain (for the ideal speedup)."""
    f = 4
    if seq == "bicgk":
        m, n = size
        return f * (2 * m * n + 2 * (m + n))
    if seq == "gemver":
        n = size                                     # GER, GER in place, GEMVT, AXPBY, GEMV
        return f * (6 * n * n + 11 * n)
    if seq == "gesummv":
        n = size
        return f * (2 * n * n + 7 * n)
    if seq == "atax":
        m, n = size
        return f * (2 * m * n + 2 * n + 2 * m)
    if seq == "axpydot":
        return f * (5 * size + 1)                    # AXPBY (w, v in; z out), DOT (z, u in; r out)
    if seq == "waxpby":
        return f * 5 * size
    raise KeyError(seq)


def algorithmic_flops(seq: str, size) -> int:
    if seq == "bicgk":
        m, n = size
        return 4 * m * n
    if seq == "gemver":
        return 8 * size * size
    if seq == "gesummv":
        return 4 * size * size
    if seq == "atax":
        m, n = size
        return 4 * m * n
    if seq == "axpydot":
        return 4 * size
    if seq == "waxpby":
        return 3 * size
    raise KeyError(seq)


# ---------------------------------------------------------------- suite

class Suite:
    """Device-resident inputs and outputs of every sequence, plus the calls."""

    def __init__(self, kf, sizes, device, seed=0, seqs=None):
        self.kf = kf
        self.sizes = sizes
        seqs = SEQS if seqs is None else seqs
        d = device
        g = lambda shape, tid: synth.uniform(shape, seed, tid, device=d)  # noqa: E731
        self.mat_ws = kf.workspace(kf.KF_SEQ_BICGK, 16384, 16384)
        if "bicgk" in seqs:
            self._mk_bicgk(kf, sizes, d, g)
        if "gemver" in seqs:
            self._mk_gemver(kf, sizes, d, g)
        if "gesummv" in seqs:
            self._mk_gesummv(kf, sizes, d, g)
        if "atax" in seqs:
            self._mk_atax(kf, sizes, d, g)
        if "axpydot" in seqs:
            self._mk_axpydot(kf, sizes, d, g)
        if "waxpby" in seqs:
            self._mk_waxpby(kf, sizes, d, g)

    def _mk_bicgk(self, kf, sizes, d, g):
        m, n = sizes["bicgk"]
        self.bicgk = dict(A=g((m, n), synth.TID["A"]), p=g((n,), synth.TID["p"]), r=g((m,), synth.TID["r"]),
                          q=torch.empty(m, device=d), s=torch.empty(n, device=d),
                          ws=kf.workspace(kf.KF_SEQ_BICGK, m, n))

    def _mk_gemver(self, kf, sizes, d, g):
        n = sizes["gemver"]
        self.gemver = dict(A=g((n, n), synth.TID["A"]), **{k: g((n,), synth.TID[k]) for k in
                                                         ("u1", "v1", "u2", "v2", "y", "z")},
                           B=torch.empty(n, n, device=d), x=torch.empty(n, device=d),
                           w=torch.empty(n, device=d), t=torch.empty(n, device=d),
                           ws=kf.workspace(kf.KF_SEQ_GEMVER, n, n))

    def _mk_gesummv(self, kf, sizes, d, g):
        n = sizes["gesummv"]
        self.gesummv = dict(A=g((n, n), synth.TID["A"]), B=g((n, n), synth.TID["B"]), x=g((n,), synth.TID["x"]),
                            y=torch.empty(n, device=d), t1=torch.empty(n, device=d),
                            t2=torch.empty(n, device=d), ws=kf.workspace(kf.KF_SEQ_GESUMMV, n, n))

    def _mk_atax(self, kf, sizes, d, g):
        m, n = sizes["atax"]
        self.atax = dict(A=g((m, n), synth.TID["A"]), x=g((n,), synth.TID["x"]), y=torch.empty(n, device=d),
                         t=torch.empty(m, device=d), ws=kf.workspace(kf.KF_SEQ_ATAX, m, n))

    def _mk_axpydot(self, kf, sizes, d, g):
        n = sizes["axpydot"]
        self.axpydot = dict(w=g((n,), synth.TID["w"]), v=g((n,), synth.TID["v"]), u=g((n,), synth.TID["u"]),
                            z=torch.empty(n, device=d), r=torch.empty(1, device=d),
                            ws=kf.workspace(kf.KF_SEQ_AXPYDOT, 1, n))

    def _mk_waxpby(self, kf, sizes, d, g):
        n = sizes["waxpby"]
        self.waxpby = dict(x=g((n,), synth.TID["x"]), y=g((n,), synth.TID["y"]), w=torch.empty(n, device=d),
                           t=torch.empty(n, device=d))

    # fused: the kernels the library emits for each canonical script
    def fused(self, seq, st):
        kf = self.kf
        if seq == "bicgk":
            b = self.bicgk
            kf.kf_bicgk(b["A"], b["p"], b["r"], b["q"], b["s"], b["ws"], stream=st)
        elif seq == "gemver":
            b = self.gemver
            kf.kf_gemver(b["A"], b["u1"], b["v1"], b["u2"], b["v2"], b["y"], b["z"], ALPHA, BETA,
                         b["B"], b["x"], b["w"], b["ws"], stream=st)
        elif seq == "gesummv":
            b = self.gesummv
            kf.kf_gesummv(b["A"], b["B"], b["x"], ALPHA, BETA, b["y"], b["ws"], stream=st)
        elif seq == "atax":
            b = self.atax
            kf.kf_atax(b["A"], b["x"], b["y"], b["ws"], stream=st)
        elif seq == "axpydot":
            b = self.axpydot
            kf.kf_axpydot(b["w"], b["v"], b["u"], ALPHA, b["z"], b["r"], b["ws"], stream=st)
        elif seq == "waxpby":
            b = self.waxpby
            kf.kf_waxpby(ALPHA, b["x"], BETA, b["y"], b["w"], stream=st)

    # unfused: one out-of-place kernel per call of the canonical script
    def unfused(self, seq, st):
        kf = self.kf
        W = self.mat_ws
        if seq == "bicgk":
            b = self.bicgk
            kf.kf_gemv(b["A"], b["p"], b["q"], W, stream=st)
            kf.kf_gemvt(b["A"], b["r"], b["s"], W, stream=st)
        elif seq == "gemver":
            b = self.gemver
            kf.kf_ger(b["A"], b["u1"], b["v1"], b["B"], stream=st)
            kf.kf_ger(b["B"], b["u2"], b["v2"], b["B"], stream=st)
            kf.kf_gemvt(b["B"], b["y"], b["t"], W, stream=st)
            kf.kf_axpby(BETA, b["t"], 1.0, b["z"], b["x"], stream=st)
            kf.kf_gemv(b["B"], b["x"], b["w"], W, alpha=ALPHA, stream=st)
        elif seq == "gesummv":
            b = self.gesummv
            kf.kf_gemv(b["A"], b["x"], b["t1"], W, alpha=ALPHA, stream=st)
            kf.kf_gemv(b["B"], b["x"], b["t2"], W, alpha=BETA, stream=st)
            kf.kf_axpby(1.0, b["t1"], 1.0, b["t2"], b["y"], stream=st)
        elif seq == "atax":
            b = self.atax
            kf.kf_gemv(b["A"], b["x"], b["t"], W, stream=st)
            kf.kf_gemvt(b["A"], b["t"], b["y"], W, stream=st)
        elif seq == "axpydot":
            b = self.axpydot
            kf.kf_axpby(1.0, b["w"], -ALPHA, b["v"], b["z"], stream=st)
            kf.kf_dot(b["z"], b["u"], b["r"], b["ws"], stream=st)
        elif seq == "waxpby":
            b = self.waxpby
            kf.kf_scal(ALPHA, b["x"], b["t"], stream=st)
            kf.kf_axpby(BETA, b["y"], 1.0, b["t"], b["w"], stream=st)

    FUSED_LAUNCHES = dict(bicgk=1, gemver=2, gesummv=1, atax=2, axpydot=1, waxpby=1)

    def inputs(self, seq):
        d = getattr(self, seq)
        keys = dict(bicgk=["A", "p", "r"], gemver=["A", "u1", "v1", "u2", "v2", "y", "z"],
                    gesummv=["A", "B", "x"], atax=["A", "x"], axpydot=["w", "v", "u"], waxpby=["x", "y"])[seq]
        return [d[k] for k in keys]

    def outputs(self, seq):
        d = getattr(self, seq)
        keys = dict(bicgk=["q", "s"], gemver=["B", "x", "w"], gesummv=["y"], atax=["y"],
                    axpydot=["z", "r"], waxpby=["w"])[seq]
        return [d[k] for k in keys]


SEQS = ["bicgk", "gemver", "gesummv", "atax", "axpydot", "waxpby"]
# the kernel the roofline names when a sequence is the first of a run
DOMINANT_KERNEL = {
    "bicgk": "matprog_kernel (BiCGK q=Ap, s=A^T r, one pass over A)",
    "gemver": "GEMVER (single cooperative launch or two matrix passes, by first-use tuning)",
    "gesummv": "matprog_kernel (GESUMMV y = alpha A x + beta B x, one pass over A and B)",
    "atax": "atax_rows_kernel + atax_finish_kernel (y = A^T (A x), one read of A)",
    "axpydot": "vecprog_kernel (AXPYDOT)",
    "waxpby": "vecprog_kernel (WAXPBY)",
}


def cached_form(kf, key):
    """The form (1 = one launch, 2 = two) the tuning cache holds for `key`
    ("gemver_form b" or "sgemvt_form bm bn"), 2 when it holds none."""
    import tempfile
    key = key + " : "
    fd, path = tempfile.mkstemp(suffix=".txt")
    os.close(fd)
    try:
        kf.kf_tune_cache_save(path)
        for line in open(path):
            if line.startswith(key):
                return 1 if line[len(key):].split()[0] == "1" else 2
    finally:
        os.unlink(path)
    return 2


def fused_launches(kf, seq, sizes):
    """Kernel launches of one fused call of `seq`.  GEMVER takes one launch
    when its first-use tuning chose the single cooperative launch (the tuning
    cache's "gemver_form" entry for the size class is 1), else two."""
    if seq != "gemver":
        return Suite.FUSED_LAUNCHES[seq]
    return cached_form(kf, f"gemver_form {sizes['gemver'].bit_length() - 1}")


# ---------------------------------------------------------------- cuBLAS context

class CublasChain:
    """The paper's comparison system on this GPU: each canonical script as
    the chain of cuBLAS calls a BLAS user writes (Section 5 compares the
    fused kernels with such CUBLAS chains), called through ctypes on the
    cuBLAS that torch loaded.  Context only, never part of the library.

    A row-major m x n matrix with lda = n is cuBLAS's column-major n x m
    matrix C = A^T, so A p is gemv(T) on C and A^T r is gemv(N) on C, and
    B += u v^T is ger(v, u) on C.  Scalars live on the device (pointer mode
    device), so no call waits for the host."""
    OP_N, OP_T = 0, 1

    def __init__(self, suite, st):
        d = torch.device("cuda", torch.cuda.current_device())
        torch.mv(torch.ones(2, 2, device=d), torch.ones(2, device=d))  # torch loads its cuBLAS
        path = None
        with open("/proc/self/maps") as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 6 and os.path.basename(parts[-1]).startswith("libcublas.so"):
                    path = parts[-1]
                    break
        self.library = os.path.basename(path) if path else "libcublas.so"
        lib = ctypes.CDLL(path or "libcublas.so")
        P, I = ctypes.c_void_p, ctypes.c_int

        def fn(name, *argtypes):
            f = getattr(lib, name)
            f.argtypes = list(argtypes)
            f.restype = ctypes.c_int
            return f

        self._create = fn("cublasCreate_v2", ctypes.POINTER(P))
        self._destroy = fn("cublasDestroy_v2", P)
        self._stream = fn("cublasSetStream_v2", P, P)
        self._pmode = fn("cublasSetPointerMode_v2", P, I)
        self._gemv = fn("cublasSgemv_v2", P, I, I, I, P, P, I, P, I, P, P, I)
        self._ger = fn("cublasSger_v2", P, I, I, P, P, I, P, I, P, I)
        self._copy = fn("cublasScopy_v2", P, I, P, I, P, I)
        self._axpy = fn("cublasSaxpy_v2", P, I, P, P, I, P, I)
        self._scal = fn("cublasSscal_v2", P, I, P, P, I)
        self._dot = fn("cublasSdot_v2", P, I, P, I, P, I, P)
        self.h = P()
        self._ok(self._create(ctypes.byref(self.h)), "cublasCreate")
        self._ok(self._stream(self.h, P(st.cuda_stream)), "cublasSetStream")
        self._ok(self._pmode(self.h, 1), "cublasSetPointerMode")
        self.sc = torch.tensor([1.0, 0.0, ALPHA, BETA, -ALPHA], device=d)
        self.suite = suite
        self.out = {}
        for seq in SEQS:
            if hasattr(suite, seq):
                self.out[seq] = [torch.empty_like(t) for t in suite.outputs(seq)]
        self.tmp = {seq: torch.empty_like(getattr(suite, seq)["t"]) for seq in ("atax",) if hasattr(suite, seq)}

    @staticmethod
    def _ok(rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} returned cuBLAS status {rc}")

    def _s(self, i):
        return self.sc.data_ptr() + 4 * i

    def run(self, seq):
        """Issue the chain of `seq` on the handle's stream."""
        one, zero, al, be, nal = (self._s(i) for i in range(5))
        b = getattr(self.suite, seq)
        o = [t.data_ptr() for t in self.out[seq]]
        h, ok = self.h, self._ok
        if seq == "bicgk":
            m, n = b["A"].shape
            ok(self._gemv(h, self.OP_T, n, m, one, b["A"].data_ptr(), n, b["p"].data_ptr(), 1, zero, o[0], 1), "gemv")
            ok(self._gemv(h, self.OP_N, n, m, one, b["A"].data_ptr(), n, b["r"].data_ptr(), 1, zero, o[1], 1), "gemv")
        elif seq == "gemver":
            n = b["A"].shape[0]
            B, x, w = o
            ok(self._copy(h, n * n, b["A"].data_ptr(), 1, B, 1), "copy")
            ok(self._ger(h, n, n, one, b["v1"].data_ptr(), 1, b["u1"].data_ptr(), 1, B, n), "ger")
            ok(self._ger(h, n, n, one, b["v2"].data_ptr(), 1, b["u2"].data_ptr(), 1, B, n), "ger")
            ok(self._copy(h, n, b["z"].data_ptr(), 1, x, 1), "copy")
            ok(self._gemv(h, self.OP_N, n, n, be, B, n, b["y"].data_ptr(), 1, one, x, 1), "gemv")
            ok(self._gemv(h, self.OP_T, n, n, al, B, n, x, 1, zero, w, 1), "gemv")
        elif seq == "gesummv":
            n = b["A"].shape[0]
            ok(self._gemv(h, self.OP_T, n, n, al, b["A"].data_ptr(), n, b["x"].data_ptr(), 1, zero, o[0], 1), "gemv")
            ok(self._gemv(h, self.OP_T, n, n, be, b["B"].data_ptr(), n, b["x"].data_ptr(), 1, one, o[0], 1), "gemv")
        elif seq == "atax":
            m, n = b["A"].shape
            t = self.tmp["atax"].data_ptr()
            ok(self._gemv(h, self.OP_T, n, m, one, b["A"].data_ptr(), n, b["x"].data_ptr(), 1, zero, t, 1), "gemv")
            ok(self._gemv(h, self.OP_N, n, m, one, b["A"].data_ptr(), n, t, 1, zero, o[0], 1), "gemv")
        elif seq == "axpydot":
            n = b["w"].numel()
            z, r = o
            ok(self._copy(h, n, b["w"].data_ptr(), 1, z, 1), "copy")
            ok(self._axpy(h, n, nal, b["v"].data_ptr(), 1, z, 1), "axpy")
            ok(self._dot(h, n, z, 1, b["u"].data_ptr(), 1, r), "dot")
        elif seq == "waxpby":
            n = b["x"].numel()
            w = o[0]
            ok(self._copy(h, n, b["y"].data_ptr(), 1, w, 1), "copy")
            ok(self._scal(h, n, be, w, 1), "scal")
            ok(self._axpy(h, n, al, b["x"].data_ptr(), 1, w, 1), "axpy")

    def outputs(self, seq):
        return self.out[seq]

    def close(self):
        if self.h:
            self._destroy(self.h)
            self.h = ctypes.c_void_p()


CUBLAS_CALLS = dict(bicgk="gemv(T), gemv(N)", gemver="copy, ger, ger, copy, gemv(N), gemv(T)",
                    gesummv="gemv(T), gemv(T)", atax="gemv(T), gemv(N)", axpydot="copy, axpy, dot",
                    waxpby="copy, scal, axpy")


def cublas_section(suite, st, steps, warmup, seqs, fused_ms):
    """Each sequence as a cuBLAS chain on the same inputs and GPU: mean ms
    (back-to-back calls between one event pair), the fused kernel's speedup
    over it, and how far its results are from the fused ones (normwise)."""
    try:
        cb = CublasChain(suite, st)
    except (OSError, AttributeError, RuntimeError) as e:
        return {"unavailable": f"cuBLAS not callable here: {e}"}
    out = {"library": cb.library, "note": "context: the paper's comparison system (CUBLAS chains) on this GPU"}
    try:
        for seq in seqs:
            ms = time_calls(lambda _st, q=seq: cb.run(q), steps, warmup, st)
            torch.cuda.synchronize()
            suite.fused(seq, st)
            torch.cuda.synchronize()
            diff = max(rel_diff(a, b) for a, b in zip(cb.outputs(seq), suite.outputs(seq)))
            out[seq] = {"calls": CUBLAS_CALLS[seq], "ms": ms, "gbs_algorithmic": algorithmic_bytes(seq, suite.sizes[seq]) / (ms * 1e-3) / 1e9,
                        "fused_speedup": ms / fused_ms[seq], "max_rel_diff_vs_fused": diff}
    finally:
        cb.close()
    return out


# ---------------------------------------------------------------- helpers

def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


DIGEST_FILES = ("matprog.cu", "matprog_impl.cuh", "matprog_f32sig.cu", "kf_device.cuh", "kf_internal.h")


def kernel_digest() -> str:
    """Digest of the sources of the BiCGK matrix pass (kernel template, its
    instances, launch geometry)."""
    h = hashlib.sha256()
    for f in DIGEST_FILES:
        with open(os.path.join(ROOT, "paper_1305_1183_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic():
    """DRAM bytes per launch of the BiCGK matrix pass from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "matprog_bicgk_16384.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    mt = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", txt)
    md = re.search(r"kernel_source_digest:\s*([0-9a-f]+)", txt)
    if not mt or not md or md.group(1) != kernel_digest():
        return None
    return int(mt.group(1))


class ClockSampler:
    """nvidia-smi sampled every 100 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- timing

def time_suite(suite, mode, steps, warmup, st, seqs):
    """Warm up, then time `steps` passes of the suite on `st`.

    Returns (total ms, {sequence: mean ms}).  The total comes from one pair
    of CUDA events around the `steps` passes, issued back to back as a user
    would (consecutive kernels may overlap their launch through programmatic
    dependent launch); each sequence's mean comes from one event pair around
    `steps` back-to-back calls of that sequence alone."""
    call = suite.fused if mode == "fused" else suite.unfused
    torch.cuda.synchronize()  # inputs come from other streams
    with torch.cuda.stream(st):
        for _ in range(warmup):
            for s in seqs:
                call(s, st)
    st.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        t0.record(st)
        for k in range(steps):
            for s in seqs:
                call(s, st)
        t1.record(st)
    st.synchronize()
    total_ms = t0.elapsed_time(t1)
    per = {}
    for s in seqs:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            a.record(st)
            for k in range(steps):
                call(s, st)
            b.record(st)
        st.synchronize()
        per[s] = a.elapsed_time(b) / steps
    return total_ms, per


def time_e2e(suite, steps, warmup, st, seqs):
    """Same metric through the public API from pinned host buffers: every step
    copies the inputs host->device, runs the fused suite and reads the results
    back device->host."""
    hin = {s: [t.detach().cpu().pin_memory() for t in suite.inputs(s)] for s in seqs}
    hout = {s: [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in suite.outputs(s)] for s in seqs}
    h2d = sum(t.numel() * t.element_size() for s in seqs for t in hin[s])
    d2h = sum(t.numel() * t.element_size() for s in seqs for t in hout[s])

    def one():
        for s in seqs:
            for dst, src in zip(suite.inputs(s), hin[s]):
                dst.copy_(src, non_blocking=True)
            suite.fused(s, st)
            for dst, src in zip(hout[s], suite.outputs(s)):
                dst.copy_(src, non_blocking=True)

    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        for _ in range(warmup):
            one()
    st.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        a.record(st)
        for _ in range(steps):
            one()
        b.record(st)
    st.synchronize()
    return a.elapsed_time(b), h2d, d2h


def time_e2e_pipelined(kf, sizes, device, steps, warmup, seqs):
    """The end-to-end metric with copies overlapped across steps: two device
    copies of the suite's buffers; step k copies its inputs host->device on
    one stream (into copy k % 2, once the kernels of step k - 2 are done
    with it), runs the fused suite on a second stream, and reads its results
    back device->host on a third, so the copies of step k + 1 overlap the
    kernels and read-back of step k.  Every step still moves all of its
    inputs in and all of its results out.  Returns (ms per step, h2d bytes,
    d2h bytes)."""
    suites = [Suite(kf, sizes, device, seqs=seqs) for _ in range(2)]
    hin = {s: [t.detach().cpu().pin_memory() for t in suites[0].inputs(s)] for s in seqs}
    hout = {s: [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in suites[0].outputs(s)] for s in seqs}
    h2d = sum(t.numel() * t.element_size() for s in seqs for t in hin[s])
    d2h = sum(t.numel() * t.element_size() for s in seqs for t in hout[s])
    s_in, s_run, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()  # noqa: E731
    loaded = [ev(), ev()]
    ran = [ev(), ev()]
    read = [ev(), ev()]
    used = [False, False]

    def step(k):
        b = k % 2
        su = suites[b]
        with torch.cuda.stream(s_in):
            if used[b]:
                s_in.wait_event(ran[b])           # step k - 2's kernels are done with copy b
            for s in seqs:
                for dst, src in zip(su.inputs(s), hin[s]):
                    dst.copy_(src, non_blocking=True)
            loaded[b].record(s_in)
        with torch.cuda.stream(s_run):
            s_run.wait_event(loaded[b])
            if used[b]:
                s_run.wait_event(read[b])         # step k - 2's results are read back
            for s in seqs:
                su.fused(s, s_run)
            ran[b].record(s_run)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ran[b])
            for s in seqs:
                for dst, src in zip(hout[s], su.outputs(s)):
                    dst.copy_(src, non_blocking=True)
            read[b].record(s_out)
        used[b] = True

    torch.cuda.synchronize()
    for k in range(warmup):
        step(k)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    z = torch.cuda.Event(enable_timing=True)
    a.record(s_in)
    for k in range(warmup, warmup + steps):
        step(k)
    s_in.wait_stream(s_out)
    s_in.wait_stream(s_run)
    z.record(s_in)
    torch.cuda.synchronize()
    ms = a.elapsed_time(z) / steps
    del suites
    torch.cuda.empty_cache()
    return ms, h2d, d2h


# ---------------------------------------------------------------- Table 1 sequences beyond the suite

def table1_bytes(seq, n):
    """Algorithmic and unfused-chain bytes of the other Table 1 sequences
    (FP32): SGEMV z = alpha A x + beta y; SGEMVT x = beta A^T y + z,
    w = alpha A x (A read twice: w needs all of x); SSCAL x = alpha x;
    MADD C = A + B; VADD x = w + y + z."""
    f = 4
    if seq == "sgemv":
        return f * (n * n + 3 * n), f * (n * n + 5 * n)           # GEMV then AXPBY
    if seq == "sgemvt":
        return f * (2 * n * n + 5 * n), f * (2 * n * n + 7 * n)   # GEMVT, AXPBY, GEMV
    if seq == "sscal":
        return f * 2 * n, f * 2 * n                                # one call either way
    if seq == "madd":
        return f * 3 * n * n, f * 3 * n * n
    if seq == "vadd":
        return f * 4 * n, f * 6 * n                                # two AXPBYs
    raise KeyError(seq)


def table1_section(kf, d, st, steps, warmup, n_mat=8192, n_vec=1 << 26):
    """SGEMV, SGEMVT, SSCAL, MADD and VADD of Table 1 (the sequences beyond
    the at-scale suite), each fused against its one-kernel-per-call chain on
    the same inputs: mean ms of back-to-back calls, GB/s of algorithmic
    bytes and fraction of the measured copy bandwidth."""
    g = lambda shape, tid: synth.uniform(shape, 0, tid, device=d)  # noqa: E731
    peak, _ = hbm_peak()
    n = n_mat
    A, B = g((n, n), synth.TID["A"]), g((n, n), synth.TID["B"])
    x, y, z = g((n,), synth.TID["x"]), g((n,), synth.TID["y"]), g((n,), synth.TID["z"])
    o1, o2, t = torch.empty(n, device=d), torch.empty(n, device=d), torch.empty(n, device=d)
    C = torch.empty(n, n, device=d)
    W = kf.workspace(kf.KF_SEQ_SGEMVT, n, n)
    vw, vy, vz = (g((n_vec,), synth.TID[k]) for k in ("w", "y", "z"))
    vo, vt = torch.empty(n_vec, device=d), torch.empty(n_vec, device=d)
    calls = {
        "sgemv": (lambda s: kf.kf_gemv(A, x, o1, W, alpha=ALPHA, beta=BETA, y0=y, stream=s),
                  lambda s: (kf.kf_gemv(A, x, t, W, alpha=ALPHA, stream=s),
                             kf.kf_axpby(1.0, t, BETA, y, o1, stream=s)), n, 1, 2),
        "sgemvt": (lambda s: kf.kf_sgemvt(A, y, z, ALPHA, BETA, o1, o2, W, stream=s),
                   lambda s: (kf.kf_gemvt(A, y, t, W, stream=s), kf.kf_axpby(BETA, t, 1.0, z, o1, stream=s),
                              kf.kf_gemv(A, o1, o2, W, alpha=ALPHA, stream=s)), n, 2, 3),
        "sscal": (lambda s: kf.kf_scal(ALPHA, vw, vo, stream=s), None, n_vec, 1, 1),
        "madd": (lambda s: kf.kf_madd(A, B, C, stream=s), None, n, 1, 1),
        "vadd": (lambda s: kf.kf_vadd3(vw, vy, vz, vo, stream=s),
                 lambda s: (kf.kf_axpby(1.0, vw, 1.0, vy, vt, stream=s), kf.kf_axpby(1.0, vt, 1.0, vz, vo, stream=s)),
                 n_vec, 1, 2),
    }
    out = {"note": "Table 1 sequences beyond the suite; SSCAL and MADD are one call either way"}
    for seq, (fused, unfused, size, nl_f, nl_u) in calls.items():
        alg, unf = table1_bytes(seq, size)
        ms = time_calls(fused, steps, warmup, st)
        if seq == "sgemvt":  # the form kf_sgemvt's first-use tuning chose (the call above ran it)
            b = n.bit_length() - 1
            nl_f = cached_form(kf, f"sgemvt_form {b} {b}")
        r = {"size": size, "ms": ms, "gbs": alg / (ms * 1e-3) / 1e9, "launches": nl_f}
        if seq == "sgemvt":
            ms1 = time_calls(lambda s: kf.kf_sgemvt_single(A, y, z, ALPHA, BETA, o1, o2, W, stream=s),
                             steps, warmup, st)
            r.update({"single_launch_ms": ms1, "single_launch_gbs": alg / (ms1 * 1e-3) / 1e9})
        r["frac"] = r["gbs"] / peak
        if unfused is not None:
            ums = time_calls(unfused, steps, warmup, st)
            r.update({"unfused_ms": ums, "unfused_launches": nl_u, "speedup_vs_unfused": ums / ms,
                      "ideal_speedup": unf / alg})
        out[seq] = r
    del A, B, C, vw, vy, vz, vo, vt
    torch.cuda.empty_cache()
    return out


def bicgk_small_section(kf, d, st, steps, warmup, n=2048, copies=16):
    """BiCGK on a 2048 x 2048 matrix (16.8 MB, inside the 129 MB L2): cold
    HBM (each call reads one of `copies` distinct copies of the inputs in
    turn, together more than twice the L2, so a copy is evicted before it is
    read again) and warm L2 (the same copy every call)."""
    peak, _ = hbm_peak()
    sets = []
    for c in range(copies):
        sets.append(dict(A=synth.uniform((n, n), c, synth.TID["A"], device=d),
                         p=synth.uniform((n,), c, synth.TID["p"], device=d),
                         r=synth.uniform((n,), c, synth.TID["r"], device=d),
                         q=torch.empty(n, device=d), s=torch.empty(n, device=d)))
    W = kf.workspace(kf.KF_SEQ_BICGK, n, n)
    nbytes = algorithmic_bytes("bicgk", (n, n))

    def cold(stream):
        for b in sets:
            kf.kf_bicgk(b["A"], b["p"], b["r"], b["q"], b["s"], W, stream=stream)

    def unfused_cold(stream):
        for b in sets:
            kf.kf_gemv(b["A"], b["p"], b["q"], W, stream=stream)
            kf.kf_gemvt(b["A"], b["r"], b["s"], W, stream=stream)

    b0 = sets[0]
    ms_cold = time_calls(cold, steps, warmup, st) / copies
    ms_ucold = time_calls(unfused_cold, steps, warmup, st) / copies
    ms_warm = time_calls(lambda s: kf.kf_bicgk(b0["A"], b0["p"], b0["r"], b0["q"], b0["s"], W, stream=s),
                         steps * copies, warmup, st)
    ms_uwarm = time_calls(lambda s: (kf.kf_gemv(b0["A"], b0["p"], b0["q"], W, stream=s),
                                     kf.kf_gemvt(b0["A"], b0["r"], b0["s"], W, stream=s)), steps * copies, warmup, st)
    out = {"n": n, "bytes": nbytes, "copies_rotated": copies,
           "cold_hbm": {"ms": ms_cold, "gbs": nbytes / (ms_cold * 1e-3) / 1e9,
                        "frac": nbytes / (ms_cold * 1e-3) / 1e9 / peak, "unfused_ms": ms_ucold,
                        "speedup_vs_unfused": ms_ucold / ms_cold},
           "warm_l2": {"ms": ms_warm, "gbs": nbytes / (ms_warm * 1e-3) / 1e9, "unfused_ms": ms_uwarm,
                       "speedup_vs_unfused": ms_uwarm / ms_warm}}
    del sets
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- precision forms

def time_calls(fn, steps, warmup, st):
    """Mean ms of fn(st) over `steps` runs on `st` after `warmup` runs (the
    device is idle first: work queued on other streams would overlap)."""
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        for _ in range(warmup):
            fn(st)
    st.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        a.record(st)
        for _ in range(steps):
            fn(st)
        b.record(st)
    st.synchronize()
    return a.elapsed_time(b) / steps


def read_probe_section(kf, suite, sizes, steps, warmup, st):
    """A read-only probe: the library's own dot product over two of the
    suite's long vectors (each read once, one float written), the call the
    unfused AXPYDOT chain makes, timed on its own like the sequences.  A
    failure is reported in the result; the other measurements stand."""
    pb = suite.axpydot
    n = sizes["axpydot"]
    try:
        ms = time_calls(lambda s: kf.kf_dot(pb["w"], pb["v"], pb["r"], pb["ws"], stream=s), steps, warmup, st)
        return {"gbs": (8 * n + 4) / (ms * 1e-3) / 1e9, "ms": ms, "bytes_per_launch": 8 * n + 4,
                "kernel": f"vecprog via kf_dot: x . y over two vectors of {n} floats (reads only)"}
    except Exception as e:
        return {"error": str(e)[:200]}


def rel_diff(a, b):
    """max |a - b| / max |b| (normwise difference of a result from the FP32 path's)."""
    return float((a.double() - b.double()).abs().max() / b.double().abs().max().clamp_min(1e-300))


def precision_section(kf, d, st, steps, warmup, n=16384):
    """BiCGK and GEMVER at n with A stored FP32, BF16 or FP8-E4M3 (per-row
    FP32 scales, FP32 vectors and accumulation).  GB/s counts the bytes each
    form must move (codes, scales, vectors); the error column is the
    low-precision result's normwise difference from the FP32 path's (the
    errors against the FP64 oracle are checked by the full-size tests)."""
    g = lambda shape, tid: synth.uniform(shape, 0, tid, device=d)  # noqa: E731
    A = g((n, n), synth.TID["A"])
    p, r = g((n,), synth.TID["p"]), g((n,), synth.TID["r"])
    vs = {k: g((n,), synth.TID[k]) for k in ("u1", "v1", "u2", "v2", "y", "z")}
    out = {"n": n, "bicgk": {}, "gemver": {},
           "error_reference": ("FP64 evaluation of the definitions on the original FP32 inputs (torch float64 "
                               "on the device): max |yhat - y| and max |yhat - y| / max |y| per result")}
    ref = {}
    # the FP64 results of the original FP32 problem
    with torch.no_grad():
        A64 = A.double()
        f64 = {"q": A64 @ p.double(), "s": A64.t() @ r.double()}
        d64 = {k: v.double() for k, v in vs.items()}
        A64.add_(torch.outer(d64["u1"], d64["v1"])).add_(torch.outer(d64["u2"], d64["v2"]))  # B in place
        f64["x"] = BETA * (A64.t() @ d64["y"]) + d64["z"]
        f64["w"] = ALPHA * (A64 @ f64["x"])
        del A64, d64
        torch.cuda.empty_cache()

    def errs(got, key):
        e = (got.double() - f64[key]).abs().max()
        return {"max_abs": float(e), "rel": float(e / f64[key].abs().max())}
    # FP32 paths
    q, sv = torch.empty(n, device=d), torch.empty(n, device=d)
    W = kf.workspace(kf.KF_SEQ_BICGK, n, n)
    ms = time_calls(lambda s: kf.kf_bicgk(A, p, r, q, sv, W, stream=s), steps, warmup, st)
    ref["bicgk"] = (q.clone(), sv.clone())
    b32 = 4 * (n * n + 4 * n)
    out["bicgk"]["f32"] = {"ms": ms, "gbs": b32 / (ms * 1e-3) / 1e9,
                           "error_vs_fp64": {"q": errs(q, "q"), "s": errs(sv, "s")}}
    B = torch.empty(n, n, device=d)
    x, w = torch.empty(n, device=d), torch.empty(n, device=d)
    WG = kf.workspace(kf.KF_SEQ_GEMVER, n, n)
    ms = time_calls(lambda s: kf.kf_gemver(A, vs["u1"], vs["v1"], vs["u2"], vs["v2"], vs["y"], vs["z"], ALPHA,
                                           BETA, B, x, w, WG, stream=s), steps, warmup, st)
    ref["gemver"] = (x.clone(), w.clone())
    g32 = 4 * (3 * n * n + 9 * n)
    out["gemver"]["f32"] = {"ms": ms, "gbs": g32 / (ms * 1e-3) / 1e9,
                            "error_vs_fp64": {"x": errs(x, "x"), "w": errs(w, "w")}}
    del B
    for name, kfmt, tdt, nb in (("bf16", kf.KF_BF16_ROWSCALE, torch.int16, 2),
                                ("e4m3", kf.KF_FP8E4M3_ROWSCALE, torch.uint8, 1)):
        Q = torch.empty((n, n), dtype=tdt, device=d)
        sA = torch.empty(n, device=d)
        kf.kf_quantize_rows(A, kfmt, Q, sA)
        W = kf.workspace(kf.KF_SEQ_BICGK, n, n, kfmt)
        ms = time_calls(lambda s: kf.kf_bicgk(Q, p, r, q, sv, W, fmt=kfmt, row_scale=sA, n=n, stream=s),
                        steps, warmup, st)
        by = nb * n * n + 4 * n + 4 * 4 * n
        out["bicgk"][name] = {"ms": ms, "gbs": by / (ms * 1e-3) / 1e9,
                              "speedup_vs_f32": out["bicgk"]["f32"]["ms"] / ms,
                              "q_rel_diff_vs_f32_path": rel_diff(q, ref["bicgk"][0]),
                              "s_rel_diff_vs_f32_path": rel_diff(sv, ref["bicgk"][1]),
                              "error_vs_fp64": {"q": errs(q, "q"), "s": errs(sv, "s")}}
        QB = torch.empty_like(Q)
        sB = torch.empty(n, device=d)
        WG = kf.workspace(kf.KF_SEQ_GEMVER, n, n, kfmt)
        ms = time_calls(lambda s: kf.kf_gemver_q(Q, kfmt, sA, vs["u1"], vs["v1"], vs["u2"], vs["v2"], vs["y"],
                                                 vs["z"], ALPHA, BETA, QB, sB, x, w, WG, stream=s),
                        steps, warmup, st)
        by = 3 * nb * n * n + 4 * (3 * n + 9 * n + 2 * n)
        out["gemver"][name] = {"ms": ms, "gbs": by / (ms * 1e-3) / 1e9,
                               "speedup_vs_f32": out["gemver"]["f32"]["ms"] / ms,
                               "x_rel_diff_vs_f32_path": rel_diff(x, ref["gemver"][0]),
                               "w_rel_diff_vs_f32_path": rel_diff(w, ref["gemver"][1]),
                               "error_vs_fp64": {"x": errs(x, "x"), "w": errs(w, "w")}}
        del Q, QB
    del A
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- learned planner

def learned_planner_section(device, scripts=80, ntrain=60, kmin=10, kmax=13, per_script=32, reps=3, epochs=2000):
    """A short fixed run of the learned planner: random scripts of 6-10 calls
    (AXPY, SCAL, DOT, GEMV, GEMVT, GER), timings of up to `per_script` plans
    of each training script, the cost model trained by kf_planner_train, and
    on the held-out scripts every enumerated plan timed (the exhaustive
    search) to score each method's choice by t(choice) / t(best)."""
    from paper_1305_1183_gb300 import learn
    t0 = time.time()
    res, _ = learn.run(seed=0, scripts=scripts, ntrain=ntrain, kmin=kmin, kmax=kmax, per_script=per_script,
                       reps=reps, epochs=epochs, top_k=3, device=device, log=None)
    names = {"mlp": "learned model, first choice (no timing)", "mlp_topk": "learned model, top 3 re-timed",
             "mlp_top2k": "learned model, top 6 re-timed",
             "mlp_margin": "learned model, top 3 and scores within 0.1 re-timed",
             "analytic": "analytic predictor max(t_t, t_c) + launch cost", "greedy": "fewest kernels",
             "unfused": "one kernel per call"}
    return {"config": res["config"], "seconds": round(time.time() - t0, 1),
            "test": {names.get(k, k): v for k, v in res["test"].items()},
            "plans_timed_per_test_script": res["timed_per_script"],
            "plans_per_test_script": res["test_plans_per_script"],
            "train_plans_timed": res["train_plans_timed"]}


# ---------------------------------------------------------------- batched form

def batched_shapes(count=4096, lo=32, hi=2048):
    """(m_i, n_i), each log-uniform in [lo, hi] (seeded)."""
    ms_ = synth.log_uniform_int(lo, hi, 0, synth.TID["sizes"], count).tolist()
    ns_ = synth.log_uniform_int(lo, hi, 1, synth.TID["sizes"], count).tolist()
    return list(zip(ms_, ns_))


def make_batched(kind, d, shapes, aligned=False):
    """Instances packed back to back (matrices with lda = n, or with rows
    padded to a multiple of 4 floats so that every row starts 16-byte
    aligned; vectors in four long buffers) with their descriptors: (descs,
    views, buffers, algorithmic bytes, counted on m x n, not on the padding).
    views[i] = (A_i, B_i or None, x_i, r_i, y_i, s_i)."""
    ldas = [(n + 3) // 4 * 4 if aligned else n for m, n in shapes]
    offs, tot, vm, vn, tm, tn = [], 0, [], [], 0, 0
    for (m, n), ld in zip(shapes, ldas):
        offs.append(tot); vm.append(tm); vn.append(tn)
        tot += m * ld; tm += m; tn += n
    A = synth.uniform((max(tot, 1),), 0, synth.TID["A"], device=d)
    Bm = synth.uniform((max(tot, 1),), 0, synth.TID["B"], device=d) if kind == "gesummv" else None
    X = synth.uniform((max(tn, 1),), 0, synth.TID["x"], device=d)
    R = synth.uniform((max(tm, 1),), 0, synth.TID["r"], device=d)
    Y = torch.empty(max(tm, 1), device=d)
    S = torch.empty(max(tn, 1), device=d)
    descs, views = [], []
    for i, (m, n) in enumerate(shapes):
        ld = ldas[i]
        a = A[offs[i]:offs[i] + m * ld].view(m, ld)[:, :n]
        b = Bm[offs[i]:offs[i] + m * ld].view(m, ld)[:, :n] if Bm is not None else None
        x, r = X[vn[i]:vn[i] + n], R[vm[i]:vm[i] + m]
        y, sv = Y[vm[i]:vm[i] + m], S[vn[i]:vn[i] + n]
        dd = {"m": m, "n": n, "lda": ld, "A": a.data_ptr(), "x": x.data_ptr(), "r": r.data_ptr(),
              "y": y.data_ptr(), "s": sv.data_ptr(), "alpha": ALPHA, "beta": BETA}
        if b is not None:
            dd["B"] = b.data_ptr()
        descs.append(dd)
        views.append((a, b, x, r, y, sv))
    if kind == "bicgk":
        nbytes = sum(4 * (m * n + 2 * (m + n)) for m, n in shapes)
    else:
        nbytes = sum(4 * (2 * m * n + m + n) for m, n in shapes)
    return descs, views, (A, Bm, X, R, Y, S), nbytes


def batched_section(kf, d, st, steps, warmup, count=4096, lo=32, hi=2048):
    """`count` independent BiCGK and GESUMMV instances, m and n each
    log-uniform in [lo, hi], matrices packed back to back (lda = n) with
    offset tables: one persistent launch replayed from a CUDA graph, tile
    height from the library's autotuner, against the same fused kernel
    launched once per instance (a stream loop, and the loop captured in a
    CUDA graph)."""
    shapes = batched_shapes(count, lo, hi)
    peak, _ = hbm_peak()
    out = {"instances": count, "m_n_range": [lo, hi], "matrix_elements": sum(m * n for m, n in shapes),
           "packing": "matrices back to back, lda = n (rows at any alignment)"}
    WB = kf.workspace(kf.KF_SEQ_BICGK, hi, hi)
    WG = kf.workspace(kf.KF_SEQ_GESUMMV, hi, hi)
    for kind in ("bicgk", "gesummv"):
        descs, views, bufs, nbytes = make_batched(kind, d, shapes)
        if kind == "bicgk":
            seq = kf.KF_SEQ_BICGK

            def one(s, v):
                kf.kf_bicgk(v[0], v[2], v[3], v[4], v[5], WB, stream=s)
        else:
            seq = kf.KF_SEQ_GESUMMV

            def one(s, v):
                kf.kf_gesummv(v[0], v[1], v[2], ALPHA, BETA, v[4], WG, stream=s)
        band, _ = kf.kf_batched_autotune(seq, descs, reps=3)
        bt = kf.Batched(seq, descs, band)
        ws = torch.zeros(max(bt.workspace_size(), 256), dtype=torch.uint8, device=d)
        bt.upload(ws)
        bt.capture(ws)
        t_graph = time_calls(lambda s: bt.replay(s), steps, warmup, st)
        loop_steps = max(1, min(steps, 3))
        t_loop = time_calls(lambda s: [one(s, v) for v in views], loop_steps, 1, st)
        t_loop_graph = None
        try:
            gph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gph, stream=st):
                for v in views:
                    one(None, v)
            t_loop_graph = time_calls(lambda s: gph.replay(), loop_steps, 1, st)
        except Exception as e:  # capture of per-instance launches is a comparison only
            out.setdefault("notes", []).append(f"{kind}: per-instance graph capture failed: {e}")
        gbs = nbytes / (t_graph * 1e-3) / 1e9
        out[kind] = {"band_rows": band, "bytes": nbytes, "ms": t_graph, "gbs": gbs, "frac": gbs / peak,
                     "per_instance_loop_ms": t_loop,
                     "per_instance_graph_ms": t_loop_graph,
                     "speedup_vs_per_instance_loop": t_loop / t_graph,
                     "speedup_vs_per_instance_graph": (t_loop_graph / t_graph) if t_loop_graph else None}
        del bt, ws, bufs, views, descs
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- CPU oracle

def oracle_sample(sizes, frac_rows: int, band: int = 0):
    """One pass of the FP64 oracle over row band ``band`` (1/frac_rows of
    every matrix's rows) and the matching slice of every vector.  Only the
    oracle calls are timed, not the input generation.  Returns (seconds,
    algorithmic bytes)."""
    import oracle
    t = 0.0
    nbytes = 0
    m, n = sizes["bicgk"]
    mr = max(1, m // frac_rows)
    rows = range(band * mr % m, band * mr % m + mr)
    A = synth.matrix_rows(m, n, rows, 0, synth.TID["A"]).numpy()
    p = synth.uniform((n,), 0, synth.TID["p"]).numpy()
    r = synth.uniform((m,), 0, synth.TID["r"]).numpy()[rows.start:rows.stop]
    c = time.perf_counter(); oracle.bicgk(A, p, r); t += time.perf_counter() - c
    nbytes += algorithmic_bytes("bicgk", (mr, n))
    n = sizes["gemver"]
    nr = max(1, n // max(1, int(np.sqrt(frac_rows))))
    A = synth.uniform((nr, nr), band, synth.TID["A"]).numpy()
    vs = [synth.uniform((nr,), band, synth.TID[k]).numpy() for k in ("u1", "v1", "u2", "v2", "y", "z")]
    c = time.perf_counter(); oracle.gemver(A, *vs, ALPHA, BETA); t += time.perf_counter() - c
    nbytes += algorithmic_bytes("gemver", nr)
    n = sizes["gesummv"]
    mr = max(1, n // frac_rows)
    rows = range(band * mr % n, band * mr % n + mr)
    A = synth.matrix_rows(n, n, rows, 0, synth.TID["A"]).numpy()
    B = synth.matrix_rows(n, n, rows, 0, synth.TID["B"]).numpy()
    x = synth.uniform((n,), 0, synth.TID["x"]).numpy()
    c = time.perf_counter(); oracle.gesummv(A, B, x, ALPHA, BETA); t += time.perf_counter() - c
    nbytes += 4 * (2 * mr * n + n + mr)
    m, n = sizes["atax"]
    mr = max(1, m // frac_rows)
    rows = range(band * mr % m, band * mr % m + mr)
    A = synth.matrix_rows(m, n, rows, 0, synth.TID["A"]).numpy()
    x = synth.uniform((n,), 0, synth.TID["x"]).numpy()
    c = time.perf_counter(); oracle.atax(A, x); t += time.perf_counter() - c
    nbytes += algorithmic_bytes("atax", (mr, n))
    nv = max(4, sizes["axpydot"] // frac_rows)
    w, v, u = (synth.uniform((nv,), band, synth.TID[k]).numpy() for k in ("w", "v", "u"))
    c = time.perf_counter(); oracle.axpydot(w, v, u, ALPHA); t += time.perf_counter() - c
    nbytes += algorithmic_bytes("axpydot", nv)
    c = time.perf_counter(); oracle.waxpby(ALPHA, w, BETA, v); t += time.perf_counter() - c
    nbytes += algorithmic_bytes("waxpby", nv)
    return t, nbytes


def _oracle_worker(args):
    """One host core's share of the all-core arm: `passes` oracle passes over
    its own row band(s); returns (seconds, bytes).  Runs in a spawned process."""
    sizes, frac_rows, band, passes = args
    import oracle
    oracle.lib()
    torch.set_num_threads(1)
    t, b = 0.0, 0
    for k in range(passes):
        dt, db = oracle_sample(sizes, frac_rows, band + k)
        t += dt
        b += db
    return t, b


def cpu_baseline(sizes, budget_s=4.0, frac_rows=16, runs=3):
    """FP64 oracle throughput on bounded samples, two arms, each the median of
    `runs` runs: one host thread (about budget_s of oracle time per run), and
    every host core (one spawned process per core, each over its own row
    bands; the arm's value is the sum of the processes' throughputs while
    they run side by side).  The oracle runs as it stands: one thread per
    process."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    single = []
    detail = None
    for _ in range(runs):
        t_total, b_total, passes = 0.0, 0, 0
        while t_total < budget_s and passes < 100:
            t, b = oracle_sample(sizes, frac_rows, passes)
            t_total += t
            b_total += b
            passes += 1
        single.append(b_total / t_total / 1e9)
        detail = (passes, b_total, t_total)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    per_proc = max(1, int(np.ceil(detail[0] / 2)))
    allc = []
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            for run in range(runs):
                res = pool.map(_oracle_worker, [(sizes, frac_rows, 1000 * run + 37 * i, per_proc)
                                                for i in range(cores)])
                allc.append(sum(b / t for t, b in res) / 1e9)
    except Exception as e:  # the single-thread arm stands on its own
        allc = []
        allc_err = str(e)[:200]
    out = {"value": float(np.median(single)), "unit": "GB/s", "cores": 1, "kind": "oracle",
           "runs": [round(v, 4) for v in single],
           "sample": (f"median of {runs} runs; each run {detail[0]} pass(es) of the FP64 C oracle (single thread) "
                      f"over 1/{frac_rows} row bands of every matrix and 1/{frac_rows} slices of every vector "
                      f"(GEMVER: a {max(1, sizes['gemver'] // int(np.sqrt(frac_rows)))}^2 block); "
                      f"{detail[1] / 1e9:.2f} GB of algorithmic traffic in {detail[2]:.1f} s; host has "
                      f"{os.cpu_count()} cores")}
    if allc:
        out["all_cores"] = {"value": float(np.median(allc)), "unit": "GB/s", "cores": cores,
                            "runs": [round(v, 4) for v in allc],
                            "sample": (f"median of {runs} runs; each run {cores} spawned processes, one per "
                                       f"core, each {per_proc} oracle pass(es) over its own row bands; value = "
                                       f"sum of the processes' throughputs")}
    else:
        out["all_cores"] = {"error": allc_err}
    return out


# ---------------------------------------------------------------- main

def slowest_rank_ms(ms: float, dist, device) -> float:
    """The longest timed region over all ranks.  Replicas run side by side,
    so the job ends when its slowest rank does."""
    if dist is None:
        return ms
    t = torch.tensor([ms], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(world: int, step_bytes: int, ms_per_step: float) -> float:
    """Whole-job throughput in GB/s: each of ``world`` replicas moves
    ``step_bytes`` per step, and a step lasts ``ms_per_step``."""
    return world * step_bytes / (ms_per_step * 1e-3) / 1e9


def run_reference(args, world, rank):
    if rank != 0:
        return
    sizes = SMALL if args.small else FULL
    import oracle
    oracle.build()
    frac = 64
    for k in range(args.warmup):
        oracle_sample(sizes, frac, k)
    t, b = 0.0, 0
    for k in range(args.steps):
        dt, db = oracle_sample(sizes, frac, args.warmup + k)
        t += dt
        b += db
    v = b / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded splitmix64 uniform[-1,1))",
        "config": {"workload": WORKLOAD, "sample": f"1/{frac} row band per step"},
        "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: the FP64 C oracle over a 1/{frac} row band of every matrix "
                                   f"and a 1/{frac} slice of every vector; single thread"},
        "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kf", choices=["kf", "reference"])
    ap.add_argument("--small", action="store_true", help="small sizes (quick check)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-unfused", action="store_true")
    ap.add_argument("--no-cublas", action="store_true", help="skip the cuBLAS-chain context section")
    ap.add_argument("--seqs", default=",".join(SEQS), help="comma-separated subset of the suite")
    ap.add_argument("--bicgk", type=int, default=0, help="square BiCGK size override (profiling)")
    ap.add_argument("--mat-tuning", default="", help="warps,vec,unroll,groups,stages for matrix passes")
    ap.add_argument("--no-precision", action="store_true", help="skip the BF16 / FP8 section")
    ap.add_argument("--autotune", type=int, default=3,
                    help="timed runs per candidate of the first-use tuning search (0: built-in defaults)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-instances section")
    ap.add_argument("--no-table1", action="store_true", help="skip SGEMV, SGEMVT, SSCAL, MADD, VADD")
    ap.add_argument("--no-small-bicgk", action="store_true", help="skip BiCGK 2048^2 cold / warm L2")
    ap.add_argument("--tune-cache", default="",
                    help="tuning cache file: loaded before the run if it exists, saved after it (profiling a "
                         "run with the tunings of an earlier one, without the search's own launches)")
    ap.add_argument("--learned-scripts", type=int, default=80,
                    help="random scripts of the learned-planner run (3/4 train, 1/4 held out; 0: skip)")
    ap.add_argument("--only", default="", choices=["", "batched", "precision", "table1"],
                    help="run only this section and print its JSON (profiling)")
    ap.add_argument("--batched-count", type=int, default=4096, help="instances per batched launch")
    ap.add_argument("--precision-n", type=int, default=16384,
                    help="matrix order of the precision section when run alone with --only precision (profiling)")
    args = ap.parse_args()
    assert args.warmup >= 0 and args.steps >= 1

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, world, rank)

    # the CPU baseline runs before any CUDA work (no process forked later)
    cpu = None
    sizes = dict(SMALL if args.small else FULL)
    if args.bicgk > 0:
        sizes["bicgk"] = (args.bicgk, args.bicgk)
    seqs = [s for s in args.seqs.split(",") if s]
    assert all(s in SEQS for s in seqs), seqs
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sizes)

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1305_1183_gb300 import _build, kf
    _build.build()
    kf.lib()

    if args.tune_cache and os.path.exists(args.tune_cache):
        kf.kf_tune_cache_load(args.tune_cache)  # tunings measured by an earlier run on this device
    if args.mat_tuning:
        kf.kf_set_matrix_tuning(*[int(v) for v in args.mat_tuning.split(",")])
    elif args.autotune > 0:
        # every kernel shape is searched on its first (warm-up) launch
        kf.kf_set_autotune(args.autotune)
    if args.only:
        d = torch.device("cuda", local)
        st = torch.cuda.Stream()
        if args.only == "batched":
            sec = batched_section(kf, d, st, args.steps, args.warmup, count=args.batched_count)
        elif args.only == "table1":
            sec = table1_section(kf, d, st, args.steps, args.warmup)
        else:
            sec = precision_section(kf, d, st, args.steps, args.warmup, n=args.precision_n)
        if rank == 0:
            print(json.dumps({args.only: sec}), flush=True)
            if args.tune_cache:
                kf.kf_tune_cache_save(args.tune_cache)
        return
    suite = Suite(kf, sizes, torch.device("cuda", local), seqs=seqs)
    st = torch.cuda.Stream()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    total_ms, per = time_suite(suite, "fused", args.steps, args.warmup, st, seqs)
    barrier()
    clk = clocks.stop()

    unf_total, unf_per = None, {}
    if not args.no_unfused:
        unf_total, unf_per = time_suite(suite, "unfused", args.steps, args.warmup, st, seqs)

    read_probe = read_probe_section(kf, suite, sizes, args.steps, args.warmup, st) if "axpydot" in seqs else None

    gemver_forms = None
    if "gemver" in seqs:
        # GEMVER's two forms on the suite's operands: two kernels chained by
        # programmatic dependent launch, and one cooperative launch
        b = suite.gemver
        try:
            ms1 = time_calls(lambda s_: kf.kf_gemver_single(b["A"], b["u1"], b["v1"], b["u2"], b["v2"], b["y"], b["z"],
                                                            ALPHA, BETA, b["B"], b["x"], b["w"], b["ws"], stream=s_),
                             args.steps, args.warmup, st)
            gb = algorithmic_bytes("gemver", sizes["gemver"])
            gemver_forms = {"single_launch_ms": ms1, "single_launch_gbs": gb / (ms1 * 1e-3) / 1e9,
                            "kf_gemver_ms": per["gemver"], "kf_gemver_gbs": gb / (per["gemver"] * 1e-3) / 1e9,
                            "note": "kf_gemver takes the form its first-use tuning measured faster"}
        except Exception as e:
            gemver_forms = {"error": str(e)[:200]}

    extra = {}
    if not args.no_cublas:
        extra["cublas_chain"] = cublas_section(suite, st, args.steps, args.warmup, seqs, per)
    if not args.small and args.bicgk == 0 and seqs == SEQS:
        del suite
        torch.cuda.empty_cache()
        if not args.no_precision:
            extra["precision"] = precision_section(kf, torch.device("cuda", local), st, args.steps, args.warmup)
        if not args.no_batched:
            extra["batched"] = batched_section(kf, torch.device("cuda", local), st, args.steps, args.warmup,
                                               count=args.batched_count)
        if not args.no_table1:
            extra["table1"] = table1_section(kf, torch.device("cuda", local), st, args.steps, args.warmup)
        if not args.no_small_bicgk:
            extra["bicgk_2048"] = bicgk_small_section(kf, torch.device("cuda", local), st, args.steps, args.warmup)
        if args.learned_scripts > 0:
            try:
                extra["learned_planner"] = learned_planner_section(
                    torch.device("cuda", local), scripts=args.learned_scripts,
                    ntrain=max(1, args.learned_scripts * 3 // 4))
            except Exception as e:  # reported, the other measurements stand
                extra["learned_planner"] = {"error": str(e)[:300]}
        suite = Suite(kf, sizes, torch.device("cuda", local), seqs=seqs)

    e2e = None
    if not args.no_e2e:
        e2e_steps = max(1, min(args.steps, 5))
        e2e_serial_ms, h2d, d2h = time_e2e(suite, e2e_steps, 1, st, seqs)
        del suite
        torch.cuda.empty_cache()
        e2e_ms_step, h2d, d2h = time_e2e_pipelined(kf, sizes, torch.device("cuda", local), max(4, e2e_steps), 2, seqs)
        e2e_ms = e2e_ms_step * e2e_steps

    step_bytes = sum(algorithmic_bytes(s, sizes[s]) for s in seqs)
    dev = torch.device("cuda", local)
    ms_step = slowest_rank_ms(total_ms, dist, dev) / args.steps
    value = job_gbs(world, step_bytes, ms_step)
    if not args.no_e2e:
        e2e_ms = slowest_rank_ms(e2e_ms, dist, dev)
    peak, peak_kind = hbm_peak()

    seqinfo = {}
    for s in seqs:
        b = algorithmic_bytes(s, sizes[s])
        g = b / (per[s] * 1e-3) / 1e9
        d = {"ms": per[s], "gbs": g, "frac": g / peak, "frac_nominal": g / NOMINAL_HBM_GBS,
             "gflops": algorithmic_flops(s, sizes[s]) / (per[s] * 1e-3) / 1e9,
             "ideal_speedup": unfused_bytes(s, sizes[s]) / b}
        if s in unf_per:
            d["unfused_ms"] = unf_per[s]
            d["unfused_gbs_algorithmic"] = b / (unf_per[s] * 1e-3) / 1e9
            d["speedup_vs_unfused"] = unf_per[s] / per[s]
        seqinfo[s] = d

    dom = "bicgk" if "bicgk" in seqs else seqs[0]
    dom_bytes = algorithmic_bytes(dom, sizes[dom])
    achieved = dom_bytes / (per[dom] * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": committed_traffic() if (not args.small and args.bicgk == 0 and dom == "bicgk") else None,
            "kernel": DOMINANT_KERNEL.get(dom, dom),
            "algorithmic_bytes_per_launch": dom_bytes, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
            if peak_kind == "measured" else "fallback 6.8 TB/s"}
    if read_probe is not None and "gbs" in read_probe:
        roof["read_probe_gbs"] = read_probe["gbs"]
        roof["frac_of_read_probe"] = achieved / read_probe["gbs"]

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded splitmix64 uniform[-1,1), seed 0)",
        "config": {"workload": WORKLOAD if (not args.small and args.bicgk == 0 and seqs == SEQS)
                   else f"subset {seqs}, sizes {[sizes[s] for s in seqs]}",
                   "l2": "inputs larger than L2 (every matrix / long vector exceeds 129 MB)",
                   "timing": ("value: one CUDA-event pair around the timed steps issued back to back; "
                              "sequences and roofline: one event pair around the same number of "
                              "back-to-back calls of each sequence alone"),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "tuning": (f"fixed {args.mat_tuning}" if args.mat_tuning else
                              f"autotuned on first use ({args.autotune} timed runs per candidate)"
                              if args.autotune > 0 else "built-in defaults"),
                   "alpha": ALPHA, "beta": BETA},
        "frac_of_peak": value / peak, "frac_of_nominal_8TBs": value / NOMINAL_HBM_GBS,
        "peak_hbm_gbs": peak, "peak_kind": peak_kind,
        "speedup_vs_unfused": (unf_total / total_ms) if unf_total else None,
        "sequences": seqinfo,
        "roofline": roof,
        "clocks": clk,
        "gpu_launches": args.steps * sum(fused_launches(kf, s, sizes) for s in seqs),
    }
    if read_probe is not None:
        line["read_probe"] = read_probe
    if gemver_forms is not None:
        line["gemver_forms"] = gemver_forms
    if not args.no_e2e:
        line["e2e"] = {"value": job_gbs(world, step_bytes, e2e_ms / e2e_steps), "unit": "GB/s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "ms_per_step": e2e_ms / e2e_steps,
                       "how": ("public API from pinned host buffers; each step copies all its inputs in and all "
                               "its results out; copies of step k+1 overlap the kernels and read-back of step k "
                               "(two device copies of the buffers, three streams)"),
                       "serial": {"value": job_gbs(world, step_bytes, e2e_serial_ms / e2e_steps),
                                  "ms_per_step": e2e_serial_ms / e2e_steps,
                                  "how": "the same steps with copies and kernels in order on one stream"}}
    line.update(extra)
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if args.tune_cache and rank == 0:
        kf.kf_tune_cache_save(args.tune_cache)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
