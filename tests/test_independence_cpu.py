"""The CUDA path and the oracle stay apart, and the product has no fallback (no GPU).

The oracle is test infrastructure: nothing in the package (Python binding,
CUDA sources, headers) may import, include or load it, and the oracle may
not use the package.  Only the seeded input generators (synth/) serve both,
and they import neither.  The binding refuses to run without the compiled
library instead of computing anything itself.
"""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1305_1183_gb300")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for nm in names:
            if nm.endswith(exts):
                yield os.path.join(d, nm)


def _imports(path):
    """Module names a Python file imports (absolute imports only)."""
    src = open(path).read()
    return set(re.findall(r"^\s*(?:from|import)\s+([A-Za-z_][\w\.]*)", src, flags=re.M))


def test_package_never_uses_the_oracle():
    for p in _files(PKG, (".py",)):
        mods = {m.split(".")[0] for m in _imports(p)}
        assert "oracle" not in mods, p
    for p in list(_files(PKG, (".cu", ".cuh", ".h", ".cpp"))) + [os.path.join(ROOT, "include", "kf.h")]:
        src = open(p).read()
        assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', src), p
        assert "kfo_" not in src and "libkf_oracle" not in src, p


def test_oracle_never_uses_the_package():
    top = os.path.join(ROOT, "oracle")
    for p in _files(top, (".py",)):
        mods = {m.split(".")[0] for m in _imports(p)}
        assert "paper_1305_1183_gb300" not in mods and "bench" not in mods, p
    src = open(os.path.join(top, "kf_oracle.c")).read()
    includes = re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', src)
    assert set(includes) <= {"math.h", "stdint.h", "string.h"}, includes


def test_generators_hold_no_method_code():
    for p in _files(os.path.join(ROOT, "synth"), (".py",)):
        mods = {m.split(".")[0] for m in _imports(p)}
        assert not mods & {"oracle", "paper_1305_1183_gb300", "bench"}, (p, mods)


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    from paper_1305_1183_gb300 import kf
    monkeypatch.setattr(kf, "_lib", None)
    monkeypatch.setattr(kf, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        kf.lib()
