"""Python binding of libgol (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
computation of its own: boards are created, stepped and read by the CUDA
library.  Loading fails with an exception if ``libgol.so`` has not been
built; there is no CPU fallback.

PyTorch is optional plumbing: ``use_torch_allocator()`` routes the
library's device allocations through the PyTorch caching allocator and
``gol_set_stream(torch_stream)`` runs the library on a PyTorch stream.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref
from typing import Iterable, Sequence

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_DIR, "libgol.so")

GOL_OK = 0
GOL_EINVAL = -1
GOL_ENOMEM = -2
GOL_ECUDA = -3
GOL_ETIMEOUT = -4
GOL_EBUSY = -5

GOL_LAYOUT_AUTO = 0
GOL_LAYOUT_PACKED = 1
GOL_LAYOUT_BYTES = 2

GOL_OPT_GENS_PER_PASS = 1
GOL_OPT_TILE_ROWS = 2
GOL_OPT_USE_GRAPHS = 3
GOL_OPT_WAIT_TIMEOUT_MS = 4
GOL_OPT_ORIENTATION = 5
GOL_OPT_CHAIN_PERMILLE = 6
GOL_OPT_PIPELINE = 7
GOL_OPT_ZERO_COPY = 8
GOL_OPT_BYTE_CLUSTER = 9
GOL_OPT_CRITICAL_PERMILLE = 10

# every symbol declared in include/gol.h
EXPORTED = (
    "gol_create", "gol_create_ex", "gol_destroy", "gol_set", "gol_get", "gol_set_packed",
    "gol_get_packed", "gol_set_packed_device", "gol_get_packed_device", "gol_set_packed_batch",
    "gol_get_packed_batch", "gol_get_packed_batch_async", "gol_get_region",
    "gol_step", "gol_step_batch", "gol_population", "gol_population_trace", "gol_population_trace_batch",
    "gol_generation", "gol_info",
    "gol_sync",
    "gol_set_stream", "gol_set_allocator", "gol_last_error", "gol_set_option", "gol_get_option",
    "gol_tune_set", "gol_tune_get", "gol_tune_reset", "gol_tune_class", "gol_board_storage", "gol_device_info",
    "gol_probe_int_throughput",
    "gol_debug_unfilled_wait", "gol_step_packed_noalloc", "gol_plan_units", "gol_kernel_launches",
)


class GolError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libgol error %d: %s" % (code, msg))
        self.code = code


_lib = None
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def load() -> ctypes.CDLL:
    """Loads libgol.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgol.so is missing (%s); build it with "
                          "`python paper_1209_4408_gb300/build.py` or __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    i64, i32, vp, sz = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "gol_create": [i64, i64, i32, P(vp)],
        "gol_create_ex": [i64, i64, i32, i32, P(vp)],
        "gol_destroy": [vp],
        "gol_set": [vp, vp, sz],
        "gol_get": [vp, vp, sz],
        "gol_set_packed": [vp, vp, sz],
        "gol_get_packed": [vp, vp, sz],
        "gol_set_packed_device": [vp, vp, sz],
        "gol_get_packed_device": [vp, vp, sz],
        "gol_set_packed_batch": [vp, sz, vp, sz],
        "gol_get_packed_batch": [vp, sz, vp, sz],
        "gol_get_packed_batch_async": [vp, sz, vp, sz],
        "gol_get_region": [vp, i64, i64, i64, i64, vp],
        "gol_step": [vp, i64],
        "gol_step_batch": [vp, vp, sz],
        "gol_population": [vp, P(ctypes.c_uint64)],
        "gol_population_trace": [vp, i64, sz, vp],
        "gol_population_trace_batch": [vp, sz, i64, sz, vp],
        "gol_generation": [vp, P(i64)],
        "gol_info": [vp, P(i64), P(i64), P(i32), P(i32)],
        "gol_sync": [vp],
        "gol_set_stream": [vp],
        "gol_set_allocator": [ALLOC_FN, FREE_FN, vp],
        "gol_last_error": [],
        "gol_set_option": [i32, i64],
        "gol_get_option": [i32, P(i64)],
        "gol_tune_set": [i64, i64, i32, i32],
        "gol_tune_get": [i64, i64, P(i32), P(i32)],
        "gol_tune_reset": [],
        "gol_tune_class": [i64, i64, P(i32), P(i32)],
        "gol_board_storage": [vp, P(i64), P(i64), P(i32)],
        "gol_device_info": [P(i32), P(i64), P(i32)],
        "gol_probe_int_throughput": [P(ctypes.c_double), P(ctypes.c_double)],
        "gol_debug_unfilled_wait": [i64],
        "gol_step_packed_noalloc": [vp, vp, i64, i64, i32, i64, vp],
        "gol_plan_units": [i64, i64, i32, i32, P(i32), ctypes.c_size_t, P(ctypes.c_size_t)],
        "gol_kernel_launches": [P(ctypes.c_uint64)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "gol_last_error" else i32
    _lib = lib
    return lib


def gol_last_error() -> str:
    return load().gol_last_error().decode()


def _check(rc: int):
    if rc != GOL_OK:
        raise GolError(rc, gol_last_error())


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------
def gol_create(rows: int, cols: int, torus: bool = True) -> int:
    h = ctypes.c_void_p()
    _check(load().gol_create(rows, cols, int(bool(torus)), ctypes.byref(h)))
    return h.value


def gol_create_ex(rows: int, cols: int, torus: bool, layout: int) -> int:
    h = ctypes.c_void_p()
    _check(load().gol_create_ex(rows, cols, int(bool(torus)), layout, ctypes.byref(h)))
    return h.value


def gol_destroy(h: int):
    _check(load().gol_destroy(h))


def gol_info(h: int):
    r, c, t, l = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
    _check(load().gol_info(h, ctypes.byref(r), ctypes.byref(c), ctypes.byref(t), ctypes.byref(l)))
    return r.value, c.value, bool(t.value), l.value


def gol_set(h: int, cells: np.ndarray):
    a = np.ascontiguousarray(cells, dtype=np.uint8)
    _check(load().gol_set(h, _ptr(a), a.size))


def gol_get(h: int, out: np.ndarray | None = None) -> np.ndarray:
    R, C, _, _ = gol_info(h)
    if out is None:
        out = np.empty((R, C), dtype=np.uint8)
    _check(load().gol_get(h, _ptr(out), out.size))
    return out


def gol_set_packed(h: int, words: np.ndarray):
    a = np.ascontiguousarray(words, dtype=np.uint64)
    _check(load().gol_set_packed(h, _ptr(a), a.size))


def gol_get_packed(h: int, out: np.ndarray | None = None) -> np.ndarray:
    R, C, _, _ = gol_info(h)
    if out is None:
        out = np.empty((R, (C + 63) // 64), dtype=np.uint64)
    _check(load().gol_get_packed(h, _ptr(out), out.size))
    return out


def gol_set_packed_device(h: int, dptr: int, nwords: int):
    _check(load().gol_set_packed_device(h, dptr, nwords))


def gol_get_packed_device(h: int, dptr: int, nwords: int):
    _check(load().gol_get_packed_device(h, dptr, nwords))


def _handles(hs) -> np.ndarray:
    if isinstance(hs, np.ndarray):
        return np.ascontiguousarray(hs, dtype=np.uint64)
    return np.array(hs, dtype=np.uint64)


def gol_set_packed_batch(hs: Sequence[int], words: np.ndarray):
    """``words``: the boards' packed states one after the other (1-D uint64)."""
    h = _handles(hs)
    a = np.ascontiguousarray(words, dtype=np.uint64).reshape(-1)
    _check(load().gol_set_packed_batch(_ptr(h), h.size, _ptr(a), a.size))


def gol_get_packed_batch(hs: Sequence[int], out: np.ndarray) -> np.ndarray:
    h = _handles(hs)
    if not (out.dtype == np.uint64 and out.flags.c_contiguous):
        raise ValueError("out must be a contiguous uint64 array")
    _check(load().gol_get_packed_batch(_ptr(h), h.size, _ptr(out), out.size))
    return out


def gol_get_packed_batch_async(hs: Sequence[int], out: np.ndarray) -> np.ndarray:
    """Queues the download of the boards into ``out`` (page-locked for the
    call not to wait); ``out`` is valid once the library's stream has run it."""
    h = _handles(hs)
    if not (out.dtype == np.uint64 and out.flags.c_contiguous):
        raise ValueError("out must be a contiguous uint64 array")
    _check(load().gol_get_packed_batch_async(_ptr(h), h.size, _ptr(out), out.size))
    return out


def gol_get_region(h: int, r0: int, c0: int, nr: int, nc: int) -> np.ndarray:
    out = np.empty((nr, nc), dtype=np.uint8)
    _check(load().gol_get_region(h, r0, c0, nr, nc, _ptr(out) if out.size else None))
    return out


def gol_step(h: int, generations: int):
    _check(load().gol_step(h, int(generations)))


def gol_step_batch(hs: Sequence[int], generations: Iterable[int]):
    hs_a = _handles(hs)
    g_a = (np.ascontiguousarray(generations, dtype=np.int64) if isinstance(generations, np.ndarray)
           else np.array(list(generations), dtype=np.int64))
    if hs_a.size != g_a.size:
        raise ValueError("handles and generation counts differ in length")
    _check(load().gol_step_batch(_ptr(hs_a), _ptr(g_a), hs_a.size))


def gol_step_packed_noalloc(d_board: int, d_spare: int, rows: int, cols: int, torus: bool,
                            generations: int, stream=None):
    """Steps the packed board at device address ``d_board`` in place, using
    ``d_spare`` (same size) as its second buffer; allocates no device memory."""
    sp = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(load().gol_step_packed_noalloc(d_board, d_spare, rows, cols, int(bool(torus)), int(generations), sp))


def gol_population(h: int) -> int:
    v = ctypes.c_uint64()
    _check(load().gol_population(h, ctypes.byref(v)))
    return v.value


def gol_population_trace(h: int, every: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    _check(load().gol_population_trace(h, int(every), int(n), _ptr(out) if n else None))
    return out


def gol_population_trace_batch(hs: Sequence[int], every: int, samples: int) -> np.ndarray:
    """uint64[len(hs), samples]: live cells of each board after every ``every`` generations."""
    h = _handles(hs)
    out = np.zeros((h.size, samples), dtype=np.uint64)
    _check(load().gol_population_trace_batch(_ptr(h), h.size, int(every), int(samples),
                                             _ptr(out) if out.size else None))
    return out


def gol_generation(h: int) -> int:
    v = ctypes.c_int64()
    _check(load().gol_generation(h, ctypes.byref(v)))
    return v.value


def gol_sync(h: int):
    _check(load().gol_sync(h))


# ---------------------------------------------------------------------------
# process settings
# ---------------------------------------------------------------------------
def gol_set_stream(stream) -> None:
    """``stream`` is a torch.cuda.Stream, a raw cudaStream_t (int) or None."""
    if stream is None:
        ptr = None
    elif isinstance(stream, int):
        ptr = stream
    else:
        ptr = stream.cuda_stream
    _check(load().gol_set_stream(ptr))


# Callback objects handed to the library stay alive for the life of the
# process: boards keep the allocator they were created with and call its free
# function when destroyed, possibly after the process-wide hook has changed.
_alloc_keep: list = []


def gol_set_allocator(alloc_fn, free_fn, ctx=None):
    """alloc_fn(size) -> int device pointer, free_fn(ptr); both None restores cudaMalloc."""
    if alloc_fn is None and free_fn is None:
        _check(load().gol_set_allocator(ALLOC_FN(), FREE_FN(), None))
        return

    def _a(size, _ctx):
        try:
            return int(alloc_fn(size))
        except Exception:   # reported to the library as an allocation failure
            return None

    def _f(ptr, _ctx):
        free_fn(ptr)

    refs = (ALLOC_FN(_a), FREE_FN(_f))
    _alloc_keep.append(refs)
    _check(load().gol_set_allocator(refs[0], refs[1], None))


def use_torch_allocator(device: int | None = None):
    """Routes libgol's device allocations through PyTorch's caching allocator
    on the library's stream and makes that the current PyTorch stream."""
    import torch

    dev = torch.cuda.current_device() if device is None else device
    stream = torch.cuda.current_stream(dev)

    def alloc(size):
        return torch.cuda.caching_allocator_alloc(size, dev, stream)

    def free(ptr):
        torch.cuda.caching_allocator_delete(ptr)

    gol_set_stream(stream)
    gol_set_allocator(alloc, free)
    return stream


def gol_set_option(key: int, value: int):
    _check(load().gol_set_option(key, int(value)))


def gol_get_option(key: int) -> int:
    v = ctypes.c_int64()
    _check(load().gol_get_option(key, ctypes.byref(v)))
    return v.value


def gol_tune_set(rows: int, cols: int, gens_per_pass: int, tile_rows: int):
    _check(load().gol_tune_set(rows, cols, gens_per_pass, tile_rows))


def gol_tune_get(rows: int, cols: int):
    k, t = ctypes.c_int(), ctypes.c_int()
    _check(load().gol_tune_get(rows, cols, ctypes.byref(k), ctypes.byref(t)))
    return k.value, t.value


def gol_tune_reset():
    _check(load().gol_tune_reset())


def gol_tune_class(rows: int, cols: int):
    r, w = ctypes.c_int(), ctypes.c_int()
    _check(load().gol_tune_class(rows, cols, ctypes.byref(r), ctypes.byref(w)))
    return r.value, w.value


def gol_board_storage(h: int):
    """(stored rows, stored words per row, transposed) of a board."""
    r, w, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    _check(load().gol_board_storage(h, ctypes.byref(r), ctypes.byref(w), ctypes.byref(t)))
    return r.value, w.value, bool(t.value)


UNIT_FIELDS = 17
UNIT_FIELD_NAMES = ("r0", "r_end", "H", "S", "w0", "U", "mode", "nnb")


def gol_plan_units(rows: int, words: int, gens_per_pass: int, tile_rows: int):
    """Units of a packed step of a board stored as rows x words (host only):
    a list of dicts with the fields of include/gol.h's unit record, the
    neighbour indices as ``nb`` and the pass cost as ``cost``."""
    lib = load()
    n = ctypes.c_size_t()
    _check(lib.gol_plan_units(rows, words, gens_per_pass, tile_rows, None, 0, ctypes.byref(n)))
    buf = (ctypes.c_int32 * (UNIT_FIELDS * max(1, n.value)))()
    _check(lib.gol_plan_units(rows, words, gens_per_pass, tile_rows, buf, n.value, ctypes.byref(n)))
    units = []
    for i in range(n.value):
        rec = buf[i * UNIT_FIELDS:(i + 1) * UNIT_FIELDS]
        u = dict(zip(UNIT_FIELD_NAMES, rec[:8]))
        u["nb"] = list(rec[8:8 + u["nnb"]])
        u["cost"] = rec[16]
        units.append(u)
    return units


def gol_device_info():
    s, l2, clk = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
    _check(load().gol_device_info(ctypes.byref(s), ctypes.byref(l2), ctypes.byref(clk)))
    return {"sm_count": s.value, "l2_bytes": l2.value, "sm_clock_khz": clk.value}


def gol_probe_int_throughput():
    ops, sec = ctypes.c_double(), ctypes.c_double()
    _check(load().gol_probe_int_throughput(ctypes.byref(ops), ctypes.byref(sec)))
    return ops.value, sec.value


def gol_kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    v = ctypes.c_uint64()
    _check(load().gol_kernel_launches(ctypes.byref(v)))
    return v.value


def gol_debug_unfilled_wait(timeout_ms: int) -> int:
    """Returns the library's status code (GOL_ETIMEOUT expected)."""
    return load().gol_debug_unfilled_wait(int(timeout_ms))


# ---------------------------------------------------------------------------
# a small object wrapper
# ---------------------------------------------------------------------------
class Board:
    """Owning wrapper of a gol_handle."""

    def __init__(self, rows: int, cols: int, torus: bool = True, layout: int = GOL_LAYOUT_AUTO):
        self.handle = None
        self.handle = gol_create_ex(rows, cols, torus, layout)
        self.rows, self.cols, self.torus, self.layout = gol_info(self.handle)
        _live_boards.add(self)

    @property
    def packed(self) -> bool:
        return self.layout == GOL_LAYOUT_PACKED

    def set(self, cells):
        gol_set(self.handle, cells)
        return self

    def get(self) -> np.ndarray:
        return gol_get(self.handle)

    def set_packed(self, words):
        gol_set_packed(self.handle, words)
        return self

    def get_packed(self) -> np.ndarray:
        return gol_get_packed(self.handle)

    def region(self, r0, c0, nr, nc) -> np.ndarray:
        return gol_get_region(self.handle, r0, c0, nr, nc)

    def step(self, generations: int = 1):
        gol_step(self.handle, generations)
        return self

    def population(self) -> int:
        return gol_population(self.handle)

    def generation(self) -> int:
        return gol_generation(self.handle)

    def sync(self):
        gol_sync(self.handle)

    def close(self):
        if self.handle:
            gol_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_batch(boards: Sequence[Board], generations: Iterable[int]):
    gol_step_batch([b.handle for b in boards], generations)


_live_boards: "weakref.WeakSet[Board]" = weakref.WeakSet()


@atexit.register
def _release_at_exit():
    """Frees boards and cached plans while Python callbacks still work."""
    if _lib is None:
        return
    for b in list(_live_boards):
        try:
            b.close()
        except Exception:
            pass
    try:
        gol_set_allocator(None, None)
    except Exception:
        pass
