"""The C-ABI library builds, loads on a machine without a GPU, and exports
every entry point include/pg.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2010_01775_gb300 import build as B
from paper_2010_01775_gb300 import pg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:pg_status|void|const char \*)\s*\*?\s*(pg_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return pg.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert {"pg_build_grid", "pg_splat_photons", "pg_reconstruct", "pg_build_cdf", "pg_sample_dirs",
            "pg_eval_pdf"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(pg.EXPORTED)  # the binding covers exactly the declared entry points


def test_status_strings(lib):
    for code in range(10):
        s = lib.pg_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert lib.pg_status_string(0) == b"ok"


def test_null_arguments_rejected_without_gpu(lib):
    assert lib.pg_build_grid(None, None, 0, None, None) == 1
    assert lib.pg_sync(None) == 1
    v = ctypes.c_uint64()
    assert lib.pg_info(None, 1, ctypes.byref(v)) == 1
    lib.pg_free(None)


def test_every_entry_point_rejects_null_handles_without_gpu(lib):
    """The convention at the top of include/pg.h: NULL contexts, handles and
    required pointers give PG_ERR_INVALID_ARG before any CUDA call (this
    machine has no GPU, so a call that reached CUDA would report
    PG_ERR_CUDA instead); destroying NULL is a no-op."""
    pointer = (ctypes.c_void_p, ctypes._Pointer)
    checked = 0
    for name in pg.EXPORTED:
        if name in ("pg_free", "pg_status_string"):
            continue
        f = getattr(lib, name)
        args = [None if isinstance(a, type) and issubclass(a, pointer) else 0 for a in f.argtypes]
        want = 0 if name in ("pg_destroy", "pg_budget_destroy") else 1
        assert f(*args) == want, name
        checked += 1
    assert checked == len(pg.EXPORTED) - 2


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/pg.h compiles as strict C99 and as C++11, and a C program that
    takes the address of every declared entry point links against libpg.so
    and runs (no entry point is called)."""
    import shutil
    import subprocess
    gcc, gxx = shutil.which("gcc"), shutil.which("g++")
    if not gcc or not gxx:
        pytest.skip("no host C compiler")
    names = sorted(_declared())
    src = tmp_path / "uses_pg.c"
    src.write_text('#include "pg.h"\n#include <stddef.h>\ntypedef void (*fn)(void);\n'
                   "static const fn entry[] = {\n" + "".join(f"  (fn){n},\n" for n in names) + "};\n"
                   "int main(void) {\n  size_t i, n = sizeof entry / sizeof entry[0];\n"
                   "  for (i = 0; i < n; ++i) if (!entry[i]) return 1;\n"
                   f"  return n == {len(names)} ? 0 : 2;\n}}\n")
    inc = os.path.join(ROOT, "include")
    libdir = os.path.dirname(pg.LIB_PATH)
    exe = tmp_path / "uses_pg"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, str(src), "-o", str(exe),
                    "-L", libdir, "-lpg", f"-Wl,-rpath,{libdir}"], check=True, capture_output=True)
    subprocess.run([gxx, "-std=c++11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, "-x", "c++", "-c",
                    str(src), "-o", str(tmp_path / "uses_pg_cxx.o")], check=True, capture_output=True)
    assert subprocess.run([str(exe)]).returncode == 0
