"""CPU checks of the C-ABI boundary: the library loads and exports every
entry point include/gol.h declares; without a GPU it refuses to compute."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "gol.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"\b(gol_[a-z_]+)\s*\(", txt))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1209_4408_gb300 import gol

    return gol.load()


def test_header_declares_the_boundary():
    syms = header_symbols()
    for name in ("gol_create", "gol_set", "gol_get", "gol_step", "gol_step_batch"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in header_symbols():
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr), name


def test_binding_covers_the_header():
    from paper_1209_4408_gb300 import gol

    assert set(gol.EXPORTED) == header_symbols()
    for name in gol.EXPORTED:
        assert callable(getattr(gol, name)), name


def test_exports_are_plain_c(lib):
    # the dynamic symbol table names the entry points unmangled
    import subprocess

    from paper_1209_4408_gb300 import gol

    out = subprocess.run(["nm", "-D", "--defined-only", gol.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(gol_[a-z_]+)$", out, flags=re.M))
    assert header_symbols() <= exported


def test_no_cpu_fallback_without_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1209_4408_gb300 import gol

    with pytest.raises(gol.GolError) as e:
        gol.gol_create(64, 64, True)
    assert e.value.code == gol.GOL_ECUDA


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1209_4408_gb300 import gol

    monkeypatch.setattr(gol, "_lib", None)
    monkeypatch.setattr(gol, "LIB_PATH", str(tmp_path / "libgol.so"))
    with pytest.raises(ImportError):
        gol.load()


C_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "gol.h"

int main(void) {
    gol_handle h = NULL;
    int rc = gol_create(64, 128, 1, &h);
    printf("create %d %s\n", rc, gol_last_error() ? "msg" : "nomsg");
    size_t n = 0;
    rc = gol_plan_units(16384, 256, 8, 64, NULL, 0, &n);
    int32_t *u = (int32_t *)malloc(n * GOL_UNIT_FIELDS * sizeof(int32_t));
    rc |= gol_plan_units(16384, 256, 8, 64, u, n, &n);
    printf("plan %d %zu %d %d %d\n", rc, n, u[0], u[1], u[5]);
    free(u);
    int k = 0, rows = 0;
    rc = gol_tune_get(1024, 1024, &k, &rows);
    printf("tune %d %d %d\n", rc, k > 0, rows > 0);
    printf("einval %d\n", gol_step(NULL, 1) == GOL_EINVAL);
    return 0;
}
"""


def test_c_program_links_and_calls_the_abi(lib, tmp_path):
    """The header compiles as strict C99 and a C program links the library
    and calls it: host-only calls answer, device calls refuse without a GPU."""
    import shutil
    import subprocess

    from paper_1209_4408_gb300 import gol

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_gol.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_gol"
    libdir = os.path.dirname(gol.LIB_PATH)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-lgol", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        assert out[0] == "create %d msg" % gol.GOL_ECUDA
    # 256 row blocks x 9 tiles; unit 0 covers rows [0, 64) and words [0, 28)
    assert out[1] == "plan 0 2304 0 64 28"
    assert out[2] == "tune 0 1 1"
    assert out[3] == "einval 1"
