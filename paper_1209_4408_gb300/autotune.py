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
