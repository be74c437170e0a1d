"""Oracle for the Game of Life generation step (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline use this package.  The product library never imports, links or
executes it, and it imports nothing from the product.

``gol_oracle.c`` holds the arithmetic (Section 1's eight-neighbour count and
its four transitions, on the wrap-around board of Section 2.2); this module
is a ctypes wrapper plus an independent unpacker for the packed layout
(bit j of word k = column 64k+j) so that packed results can be compared
cell by cell.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "gol_oracle.c")
_SO = os.path.join(_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``gol_oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32 = ctypes.c_int64, ctypes.c_int
        p8 = ctypes.c_void_p
        lib.oracle_step.argtypes = [i64, i64, i32, p8, p8]
        lib.oracle_run.argtypes = [i64, i64, i32, i64, p8, p8]
        lib.oracle_run_rows_omp.argtypes = [i64, i64, i32, i64, p8, p8, i32]
        lib.oracle_run_cols_omp.argtypes = [i64, i64, i32, i64, p8, p8, i32]
        lib.oracle_run_blocks_omp.argtypes = [i64, i64, i32, i64, p8, p8, i32, i32]
        lib.oracle_population.argtypes = [i64, i64, p8, ctypes.POINTER(ctypes.c_uint64)]
        for f in ("oracle_step", "oracle_run", "oracle_run_rows_omp", "oracle_run_cols_omp",
                  "oracle_run_blocks_omp", "oracle_population", "oracle_max_threads"):
            getattr(lib, f).restype = i32
        _lib = lib
    return _lib


def _cells(x) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.uint8)
    if a.ndim != 2:
        raise ValueError("board must be 2-D")
    return a


def _check(rc: int):
    if rc != 0:
        raise ValueError("oracle error %d" % rc)


def step(cells, torus: bool = True) -> np.ndarray:
    """One generation of ``cells`` (uint8 R x C, values 0/1)."""
    a = _cells(cells)
    out = np.empty_like(a)
    _check(_load().oracle_step(a.shape[0], a.shape[1], int(torus), a.ctypes.data, out.ctypes.data))
    return out


def run(cells, gens: int, torus: bool = True) -> np.ndarray:
    """``gens`` generations of ``cells``."""
    a = _cells(cells)
    out = np.empty_like(a)
    _check(_load().oracle_run(a.shape[0], a.shape[1], int(torus), int(gens),
                              a.ctypes.data, out.ctypes.data))
    return out


def run_rows_omp(cells, gens: int, threads: int, torus: bool = True) -> np.ndarray:
    """Section 2.1's by-row decomposition on ``threads`` OpenMP threads."""
    a = _cells(cells)
    out = np.empty_like(a)
    _check(_load().oracle_run_rows_omp(a.shape[0], a.shape[1], int(torus), int(gens),
                                       a.ctypes.data, out.ctypes.data, int(threads)))
    return out


def run_cols_omp(cells, gens: int, threads: int, torus: bool = True) -> np.ndarray:
    """Section 2.1's by-column decomposition on ``threads`` OpenMP threads."""
    a = _cells(cells)
    out = np.empty_like(a)
    _check(_load().oracle_run_cols_omp(a.shape[0], a.shape[1], int(torus), int(gens),
                                       a.ctypes.data, out.ctypes.data, int(threads)))
    return out


def run_blocks_omp(cells, gens: int, m: int, n: int, torus: bool = True) -> np.ndarray:
    """Section 2.2's m x n block decomposition on m*n OpenMP threads."""
    a = _cells(cells)
    out = np.empty_like(a)
    _check(_load().oracle_run_blocks_omp(a.shape[0], a.shape[1], int(torus), int(gens),
                                         a.ctypes.data, out.ctypes.data, int(m), int(n)))
    return out


def population(cells) -> int:
    """Number of live cells (the quantity of the paper's Table 1)."""
    a = _cells(cells)
    out = ctypes.c_uint64(0)
    _check(_load().oracle_population(a.shape[0], a.shape[1], a.ctypes.data, ctypes.byref(out)))
    return int(out.value)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def unpack_words(words, cols: int | None = None) -> np.ndarray:
    """uint64[R, W] in the packed layout -> uint8[R, 64W] (or the first
    ``cols`` columns).  Bit j of word k is column 64k + j."""
    w = np.ascontiguousarray(words, dtype=np.uint64)
    R, W = w.shape
    bits = (w[:, :, None] >> np.arange(64, dtype=np.uint64)[None, None, :]) & np.uint64(1)
    cells = bits.astype(np.uint8).reshape(R, W * 64)
    return cells if cols is None else np.ascontiguousarray(cells[:, :cols])
