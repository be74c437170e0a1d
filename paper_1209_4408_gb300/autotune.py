"""Autotuner for packed boards: picks generations per pass (K) and warp tile
rows for a board size class by timed trials, and persists the choice.

The paper's decompositions (Section 2: bars of rows, bars of columns, m x n
blocks) survive here only as candidate tile shapes: a unit of work is a bar
of full rows when a row fits in one warp (at most 32 words), otherwise a
block of up to 30 words by ``tile_rows`` rows.  Trials run the library's own
step on a scratch board of the class's shape; the table lives in the
library (``gol_tune_set``) and in a JSON file (``GOL_TUNE_CACHE`` or
``~/.cache/gol_gb300_tune.json``).
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import gol

DEFAULT_K = (4, 5, 6, 7, 8)
DEFAULT_ROWS = (8, 16, 32, 64, 128, 256, 512)


SHIPPED_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_gb300.json")


def cache_path() -> str:
    return os.environ.get("GOL_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                         "gol_gb300_tune.json"))


def time_config(rows: int, cols: int, k: int, tile_rows: int, gens: int, reps: int = 3) -> float:
    """Seconds per generation of a rows x cols torus under (k, tile_rows)."""
    import torch

    gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, k)
    gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, tile_rows)
    try:
        b = gol.Board(rows, cols, torus=True, layout=gol.GOL_LAYOUT_PACKED)
        rng = np.random.default_rng(rows * 131 + cols)
        b.set_packed(rng.integers(0, 2 ** 63, size=(rows, cols // 64), dtype=np.uint64))
        b.step(gens)                      # warm-up (plan building, first launch)
        b.sync()
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            b.step(gens)
            b.sync()
            best = min(best, time.perf_counter() - t)
        b.close()
        return best / gens
    finally:
        gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, 0)
        gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, 0)


def tune_shape(rows: int, cols: int, gens: int = 256, ks=DEFAULT_K, tile_rows=DEFAULT_ROWS) -> dict:
    """Tries every (k, tile_rows) for one shape; installs and returns the best."""
    trials = []
    for k in ks:
        for tr in tile_rows:
            if tr > rows:
                continue
            trials.append((time_config(rows, cols, k, tr, gens), k, tr))
    trials.sort()
    s, k, tr = trials[0]
    gol.gol_tune_set(rows, cols, k, tr)
    return {"rows": rows, "cols": cols, "k": k, "tile_rows": tr, "gcups": rows * cols / s / 1e9,
            "trials": [(round(rows * cols / t / 1e9, 2), kk, rr) for t, kk, rr in trials]}


def _time_batch(handles: np.ndarray, gens: np.ndarray, steps: int, warmup: int) -> float:
    """Mean seconds of one gol_step_batch of the boards (CUDA events on the
    library's stream, which must be PyTorch's current stream)."""
    import torch

    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        gol.gol_step_batch(handles, gens)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        gol.gol_step_batch(handles, gens)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) * 1e-3 / steps


def batch_classes(handles, gens) -> list:
    """Size classes of the packed boards of a batch, most work first: dicts
    with the class key, a representative stored shape (rows, cols) for
    gol_tune_set, the class's share of the batch's cell updates and its
    boards' largest generation count."""
    classes = {}
    total = 0
    for h, g in zip(handles, gens):
        srows, swords, _ = gol.gol_board_storage(int(h))
        if swords == 0:
            continue
        key = gol.gol_tune_class(srows, swords * 64)
        work = srows * swords * 64 * int(g)
        total += work
        c = classes.setdefault(key, {"key": key, "rows": srows, "cols": swords * 64, "work": 0, "boards": 0,
                                     "max_gens": 0})
        c["work"] += work
        c["boards"] += 1
        c["max_gens"] = max(c["max_gens"], int(g))
    out = sorted(classes.values(), key=lambda c: -c["work"])
    for c in out:
        c["share"] = c["work"] / max(1, total)
    return out


def tune_batch(handles, gens, classes: int = 12, tile_rows=(24, 32, 48, 64, 96, 128, 192, 256),
               ks=(5, 6, 7), steps: int = 4, warmup: int = 2, min_gain: float = 0.003) -> dict:
    """Tunes the size classes of one batch on the batch itself.  The
    planner takes the generations per pass of a launch from the board with
    the most work and each board's tile rows from its class's entry (then
    shortens the units of boards with long chains), so a class's best tile
    height depends on the rest of the batch: each of the `classes` classes
    with the most work gets, in turn, the tile height that makes the whole
    batch fastest with the others fixed (coordinate descent), then the
    class that sets the launch's generations per pass tries each K in
    `ks`.  A trial replaces the incumbent only when it is faster by more
    than `min_gain` (timing noise).  Installs the entries found
    (gol_tune_set) and returns them with the batch time before and after."""
    handles = np.ascontiguousarray(handles, dtype=np.uint64)
    gens = np.ascontiguousarray(gens, dtype=np.int64)
    cls = batch_classes(handles, gens)[:classes]
    before = _time_batch(handles, gens, steps, warmup)
    entries = {}
    for c in cls:
        k0, r0 = gol.gol_tune_get(c["rows"], c["cols"])
        entries[c["key"]] = [k0, r0]
    best_t = before
    for c in cls:
        k, r_best = entries[c["key"]]
        for tr in tile_rows:
            if tr == r_best:
                continue
            gol.gol_tune_set(c["rows"], c["cols"], k, tr)
            t = _time_batch(handles, gens, steps, warmup)
            if t < best_t * (1 - min_gain):
                best_t, r_best = t, tr
        gol.gol_tune_set(c["rows"], c["cols"], k, r_best)
        entries[c["key"]] = [k, r_best]
    # generations per pass: the launch takes the K of the board with the most work
    lead = max(zip(handles, gens), key=lambda hg: gol.gol_board_storage(int(hg[0]))[0] *
               gol.gol_board_storage(int(hg[0]))[1] * int(hg[1]))
    srows, swords, _ = gol.gol_board_storage(int(lead[0]))
    k_best, r_lead = gol.gol_tune_get(srows, swords * 64)
    for k in ks:
        if k == k_best:
            continue
        for c in cls:                        # the same K for every tuned class keeps one K per launch
            gol.gol_tune_set(c["rows"], c["cols"], k, entries[c["key"]][1])
        gol.gol_tune_set(srows, swords * 64, k, r_lead)
        t = _time_batch(handles, gens, steps, warmup)
        if t < best_t * (1 - min_gain):
            best_t, k_best = t, k
    for c in cls:
        gol.gol_tune_set(c["rows"], c["cols"], k_best, entries[c["key"]][1])
        entries[c["key"]][0] = k_best
    gol.gol_tune_set(srows, swords * 64, k_best, r_lead)
    after = _time_batch(handles, gens, steps, warmup)
    out = []
    for c in cls:
        out.append({"rows": c["rows"], "cols": c["cols"], "k": entries[c["key"]][0],
                    "tile_rows": entries[c["key"]][1], "class": list(c["key"]), "share": round(c["share"], 4),
                    "boards": c["boards"]})
    return {"entries": out, "before_s": before, "after_s": after, "lead": [int(srows), int(swords * 64)]}


def save(entries: list, path: str | None = None):
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump({"entries": [{k: e[k] for k in ("rows", "cols", "k", "tile_rows")} for e in entries]}, f,
                  indent=1)


def load(path: str | None = None) -> int:
    """Installs a saved table; returns the number of entries applied."""
    path = path or cache_path()
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        data = json.load(f)
    n = 0
    for e in data.get("entries", []):
        gol.gol_tune_set(int(e["rows"]), int(e["cols"]), int(e["k"]), int(e["tile_rows"]))
        n += 1
    return n


def load_shipped() -> int:
    """Installs the table measured on a GB300 that ships with the package."""
    return load(SHIPPED_TABLE)


def tune_classes(shapes, gens: int = 256) -> list:
    """Tunes a list of (rows, cols) shapes, one per size class."""
    return [tune_shape(r, c, gens) for r, c in shapes]
