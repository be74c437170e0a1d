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
