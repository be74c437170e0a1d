"""Seeded synthetic inputs for the Game of Life step.

This module is the one piece of code that both sides of every check use:
the oracle (``oracle/``) and the CUDA library (``paper_1209_4408_gb300``)
are both fed boards made here, and neither imports the other.  It holds
no neighbour counting and no transition rule: only random numbers,
layouts of the generated cells, and the placement of hand-written
patterns.

Random numbers come from SplitMix64 (G. Steele, D. Lea, C. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014; the
64-bit finaliser constants are the ones published with Vigna's
``splitmix64.c``).  ``sm64(x)`` is the first output of a SplitMix64
stream whose state starts at ``x``: add the golden-ratio increment,
then apply the finaliser.  Every generator below is counter based,
``value(i) = sm64(seed + i)``, so any sub-rectangle of a board can be
regenerated on its own without producing the rest.

Cell convention used everywhere: ``cells[r, c]`` in {0, 1}, row major.
Packed convention: ``words[r, k]`` is a little-endian uint64 whose bit
``j`` holds column ``64*k + j`` (least significant bit = lowest column).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def sm64(x) -> np.ndarray:
    """SplitMix64 output for state ``x`` (uint64 array or scalar)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def sm64_int(x: int) -> int:
    """Pure-Python SplitMix64, used to pin the numpy version."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def derive_seed(seed: int, index: int) -> int:
    """Seed of item ``index`` of a collection seeded by ``seed``.

    Boards of one batch draw from ``sm64(seed * 2**20 + index)`` rather
    than ``seed + index`` so that two boards never share a stretch of
    their counter streams.
    """
    return sm64_int((seed * (1 << 20) + index) & _MASK64)


def _counters(seed: int, start: int, count: int) -> np.ndarray:
    base = np.uint64((seed + start) & _MASK64)
    return np.arange(count, dtype=np.uint64) + base


def bernoulli_board(rows: int, cols: int, p: float, seed: int) -> np.ndarray:
    """uint8[rows, cols]; cell (r, c) is alive iff
    ``(sm64(seed + r*cols + c) >> 11) * 2**-53 < p``."""
    out = np.empty((rows, cols), dtype=np.uint8)
    chunk = max(1, (1 << 22) // max(cols, 1))
    for r0 in range(0, rows, chunk):
        r1 = min(rows, r0 + chunk)
        z = sm64(_counters(seed, r0 * cols, (r1 - r0) * cols))
        u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        out[r0:r1] = (u < p).reshape(r1 - r0, cols)
    return out


def bernoulli_region(rows: int, cols: int, p: float, seed: int,
                     r0: int, c0: int, nr: int, nc: int) -> np.ndarray:
    """The sub-rectangle [r0, r0+nr) x [c0, c0+nc) (indices taken mod the
    board size) of ``bernoulli_board(rows, cols, p, seed)``, computed
    without generating the rest of the board."""
    rr = (np.arange(r0, r0 + nr) % rows).astype(np.uint64)
    cc = (np.arange(c0, c0 + nc) % cols).astype(np.uint64)
    idx = rr[:, None] * np.uint64(cols) + cc[None, :]
    z = sm64(idx + np.uint64(seed & _MASK64))
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return (u < p).astype(np.uint8)


def random_words(rows: int, words: int, seed: int, out: np.ndarray | None = None,
                 row0: int = 0) -> np.ndarray:
    """uint64[rows, words] with ``word[r, k] = sm64(seed + (row0+r)*words + k)``:
    a packed board whose cells are i.i.d. Bernoulli(1/2).  ``out`` may be a
    preallocated (e.g. pinned) array; rows are generated in chunks."""
    if out is None:
        out = np.empty((rows, words), dtype=np.uint64)
    chunk = max(1, (1 << 23) // max(words, 1))
    for a in range(0, rows, chunk):
        b = min(rows, a + chunk)
        out[a:b] = sm64(_counters(seed, (row0 + a) * words, (b - a) * words)).reshape(b - a, words)
    return out


def random_words_region(words_per_row: int, seed: int, r0: int, nr: int,
                        k0: int, nk: int, rows: int) -> np.ndarray:
    """Words [r0, r0+nr) x [k0, k0+nk) (mod the board) of ``random_words``."""
    rr = (np.arange(r0, r0 + nr) % rows).astype(np.uint64)
    kk = (np.arange(k0, k0 + nk) % words_per_row).astype(np.uint64)
    idx = rr[:, None] * np.uint64(words_per_row) + kk[None, :]
    return sm64(idx + np.uint64(seed & _MASK64))


def pack_rows(cells: np.ndarray) -> np.ndarray:
    """uint8[R, C] (any C) -> uint64[R, ceil(C/64)] in the packed convention,
    the bits past column C of each row's last word zero."""
    cells = np.ascontiguousarray(cells, dtype=np.uint8)
    R, C = cells.shape
    W = (C + 63) // 64
    padded = np.zeros((R, 64 * W), dtype=np.uint8)
    padded[:, :C] = cells
    return pack_cells(padded)


def pack_cells(cells: np.ndarray) -> np.ndarray:
    """uint8[R, C] (C % 64 == 0) -> uint64[R, C/64] in the packed convention."""
    cells = np.ascontiguousarray(cells, dtype=np.uint8)
    R, C = cells.shape
    if C % 64:
        raise ValueError("pack_cells needs cols % 64 == 0")
    b = np.packbits(cells, axis=1, bitorder="little")  # R x C/8, bit j of byte i = col 8i+j
    return np.ascontiguousarray(b).view("<u8").reshape(R, C // 64).astype(np.uint64, copy=False)


def bernoulli_words(rows: int, cols: int, p: float, seed: int) -> np.ndarray:
    """``bernoulli_board`` delivered in the packed convention."""
    return pack_cells(bernoulli_board(rows, cols, p, seed))


# ---------------------------------------------------------------------------
# Hand-written patterns (standard Life objects; coordinates are (row, col)).
# ---------------------------------------------------------------------------
PATTERNS = {
    # period-4 glider travelling towards +row, +col
    "glider": [(0, 1), (1, 2), (2, 0), (2, 1), (2, 2)],
    # period-2 oscillator, horizontal phase
    "blinker": [(1, 0), (1, 1), (1, 2)],
    # still lifes
    "block": [(0, 0), (0, 1), (1, 0), (1, 1)],
    "beehive": [(0, 1), (0, 2), (1, 0), (1, 3), (2, 1), (2, 2)],
}


def place(board: np.ndarray, name: str, r: int, c: int) -> np.ndarray:
    """Set the cells of pattern ``name`` with its origin at (r, c), wrapping."""
    R, C = board.shape
    for dr, dc in PATTERNS[name]:
        board[(r + dr) % R, (c + dc) % C] = 1
    return board


def pattern_board(rows: int, cols: int, name: str, r: int = 1, c: int = 1) -> np.ndarray:
    return place(np.zeros((rows, cols), dtype=np.uint8), name, r, c)


# ---------------------------------------------------------------------------
# Workload recipes.  Seeds are 14408 + configuration number.
# ---------------------------------------------------------------------------
SEED_BYTES_256 = 14409      # 256x256 byte board, Bernoulli(0.3)
SEED_SINGLE_16K = 14410     # 16384^2 packed board, Bernoulli(0.5)
SEED_BATCH_4096 = 14411     # 4096-board batch
SEED_SERVE = 14412          # request stream
SEED_HUGE_128K = 14413      # 131072^2 board with a glider band
SEED_MASKED = 14414         # board with neither side a multiple of 64


def _round64(x: float, lo: int, hi: int) -> int:
    v = int(round(x / 64.0)) * 64
    return max(lo, min(hi, v))


@dataclass
class BoardSpec:
    index: int
    rows: int
    cols: int
    density: float
    gens: int
    seed: int

    @property
    def cells(self) -> int:
        return self.rows * self.cols


def batch_specs(n: int = 4096, seed: int = SEED_BATCH_4096, side_lo: float = 32.0,
                side_hi: float = 2048.0, gen_lo: float = 100.0, gen_hi: float = 5000.0) -> list[BoardSpec]:
    """Uneven batch: rows and cols independently log-uniform in
    [side_lo, side_hi], rounded to the nearest multiple of 64 and clamped to
    [64, side_hi]; density U(0.1, 0.6); generations round(log-uniform
    [gen_lo, gen_hi])."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n):
        r = _round64(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi))), 64, int(side_hi))
        c = _round64(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi))), 64, int(side_hi))
        d = float(rng.uniform(0.1, 0.6))
        g = int(round(math.exp(rng.uniform(math.log(gen_lo), math.log(gen_hi)))))
        specs.append(BoardSpec(i, r, c, d, g, derive_seed(seed, i)))
    return specs


@dataclass
class Request:
    index: int
    arrival_s: float
    rows: int
    cols: int
    density: float
    gens: int
    seed: int

    @property
    def work(self) -> int:
        return self.rows * self.cols * self.gens


def request_stream(n: int, rate_per_s: float, seed: int = SEED_SERVE,
                   side_lo: float = 32.0, side_hi: float = 8192.0,
                   gen_lo: float = 10.0, gen_hi: float = 1e5) -> list[Request]:
    """Poisson arrivals at ``rate_per_s``; sides log-uniform [side_lo, side_hi]
    rounded/clamped to multiples of 64 in [64, side_hi]; density U(0.1, 0.6);
    generations round(log-uniform [gen_lo, gen_hi])."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        r = _round64(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi))), 64, int(side_hi))
        c = _round64(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi))), 64, int(side_hi))
        d = float(rng.uniform(0.1, 0.6))
        g = int(round(math.exp(rng.uniform(math.log(gen_lo), math.log(gen_hi)))))
        out.append(Request(i, t, r, c, d, g, derive_seed(seed, i)))
    return out


@dataclass
class GliderBand:
    """A cleared band of ``band_rows`` full-width rows starting at ``b0`` that
    holds an ``n x n`` lattice of gliders (see ``PATTERNS['glider']``) with
    spacing ``spacing``, the first glider's origin at (b0 + off_r, off_c)."""
    b0: int = 65536
    band_rows: int = 4096
    n: int = 64
    spacing: int = 16
    off_r: int = 1280
    off_c: int = 1024

    def glider_cells(self, t: int = 0) -> np.ndarray:
        """(row, col) of all glider cells after ``t`` generations, t % 4 == 0
        (each glider has moved t/4 rows and t/4 cols)."""
        assert t % 4 == 0
        s = t // 4
        base = np.array(PATTERNS["glider"], dtype=np.int64)
        gi = np.arange(self.n, dtype=np.int64) * self.spacing
        rr = (self.b0 + self.off_r + gi[:, None, None] + base[None, None, :, 0] + s)
        cc = (self.off_c + gi[None, :, None] + base[None, None, :, 1] + s)
        rr = np.broadcast_to(rr, (self.n, self.n, len(base))).reshape(-1)
        cc = np.broadcast_to(cc, (self.n, self.n, len(base))).reshape(-1)
        return np.stack([rr, cc], axis=1)


def glider_band_words(rows: int, words: int, seed: int, band: GliderBand,
                      out: np.ndarray | None = None) -> np.ndarray:
    """Packed 131072^2-style board: Bernoulli(1/2) words everywhere, the band
    rows cleared, then the glider lattice set."""
    out = random_words(rows, words, seed, out=out)
    out[band.b0:band.b0 + band.band_rows] = 0
    rc = band.glider_cells(0)
    r, c = rc[:, 0] % rows, rc[:, 1] % (words * 64)
    np.bitwise_or.at(out, (r, c // 64), np.left_shift(np.uint64(1), (c % 64).astype(np.uint64)))
    return out
