"""The C-ABI library builds, loads and exports every declared symbol (no GPU).

Only argument validation runs here: those paths return before any CUDA call.
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "kf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(kf_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def kf():
    from paper_1305_1183_gb300 import _build, kf as K
    _build.build()
    K.lib()
    return K


def test_every_declared_symbol_is_exported(kf):
    names = declared_functions()
    assert len(names) >= 20, names
    L = kf.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding covers every declared entry point under the same name
    assert set(names) <= set(kf.exported_symbols()), set(names) - set(kf.exported_symbols())


def test_validation_without_gpu(kf):
    L = kf.lib()
    assert L.kf_bicgk(-1, 4, None, 4, 0, None, None, None, None, None, None, 0, None) == -1
    assert L.kf_bicgk(4, 4, None, 4, 0, None, None, None, None, None, None, 0, None) == -1
    assert b"null matrix" in L.kf_last_error()
    assert L.kf_bicgk(4, 8, 1024, 4, 0, None, 16, 16, 16, 16, None, 0, None) == -2   # lda < n
    assert L.kf_bicgk(4, 4, 1024, 4, 9, None, 16, 16, 16, 16, None, 0, None) == -3   # format
    assert L.kf_bicgk(4, 4, 1024, 4, 2, None, 16, 16, 16, 16, None, 0, None) == -1   # scales
    assert L.kf_set_matrix_tuning(3, 2, 2, 0, 4) == -1
    assert L.kf_set_matrix_tuning(8, 2, 2, 0, 9) == -1
    assert L.kf_set_matrix_tuning(8, 2, 2, 0, 4) == 0
    assert L.kf_set_matrix_tuning(0, 0, 0, 0, 0) == 0      # back to automatic
    assert L.kf_set_autotune(-1) == -1 and L.kf_set_autotune(101) == -1
    assert L.kf_set_autotune(0) == 0 and kf.kf_get_autotune() == 0
    b = ctypes.c_size_t(0)
    assert L.kf_workspace_size(0, 16384, 16384, 0, ctypes.byref(b)) == 0
    assert 0 < b.value < 64 << 20          # bounded, small next to the 1 GiB matrix
    assert L.kf_workspace_size(42, 1, 1, 0, ctypes.byref(b)) == -1
    assert L.kf_axpydot(10, None, None, None, 1.0, None, None, None, 0, None) == -1
    assert L.kf_ger(4, 4, 1024, 4, 1.0, 16, 16, 1024, 8, None) == -2                   # in place, ldb != lda


def test_binding_constants_match_the_header(kf):
    """Status codes and sequence ids in the Python binding equal the
    header's, name for name."""
    src = open(os.path.join(ROOT, "include", "kf.h")).read()
    codes = dict(re.findall(r"#define\s+(KF_(?:OK|ERR_\w+))\s+\(?(-?\d+)\)?", src))
    assert len(codes) >= 12, codes
    for name, v in codes.items():
        assert getattr(kf, name) == int(v), name
    seqs = re.findall(r"\b(KF_SEQ_\w+)\s*=\s*(\d+)", src)
    assert len(seqs) >= 9
    for name, v in seqs:
        assert getattr(kf, name) == int(v), name


def test_header_is_plain_c_and_links(kf, tmp_path):
    """include/kf.h compiles as strict C99 (no C++ or torch types), and a C
    program that takes the address of every declared function links
    against the library and runs (kf_version needs no device)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    names = declared_functions()
    src = tmp_path / "use_all.c"
    src.write_text('#include "kf.h"\n#include <stdio.h>\nint main(void) {\n'
                   "  typedef void (*fnp)(void);\n  const fnp fns[] = {\n"
                   + "".join(f"    (fnp)&{n},\n" for n in names)
                   + '  };\n  printf("%s|%d\\n", kf_version(), (int)(sizeof(fns) / sizeof(fns[0])));\n'
                   "  return 0;\n}\n")
    libdir = os.path.dirname(kf.library_path())
    exe = tmp_path / "use_all"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I" + os.path.join(ROOT, "include"), str(src), "-L" + libdir, "-lkf",
                        "-Wl,-rpath," + libdir, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    version, count = out.stdout.strip().split("|")
    assert version == kf.kf_version() and int(count) == len(names)


def test_readme_c_example_compiles_and_links(kf, tmp_path):
    """The C example in README.md builds against the header, the CUDA
    runtime and the library (it runs only on a GPU)."""
    import re
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if gcc is None or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("no C compiler or CUDA headers")
    block = re.search(r"```c\n(.*?)```", open(os.path.join(ROOT, "README.md")).read(), flags=re.S)
    assert block, "README has no C example"
    src = tmp_path / "example.c"
    src.write_text(block.group(1) + "\nint main(void) { return 0; }\n")
    libdir = os.path.dirname(kf.library_path())
    cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                    if os.path.exists(d)), None)
    cmd = [gcc, "-std=c99", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"),
           "-I" + os.path.join(cuda, "include"), str(src), "-L" + libdir, "-lkf", "-L" + cudalib, "-lcudart",
           "-o", str(tmp_path / "example")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
