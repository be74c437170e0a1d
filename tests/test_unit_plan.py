"""Host logic of the packed step's unit plan (no GPU needed).

A persistent launch splits each board into units (the output rectangle one
warp produces per pass: Section 2.2's spatial blocks, here row blocks times
word tiles) and orders the passes of neighbouring units by join counters.
The step is only correct if
  * the units' output cells cover the board exactly once, and
  * every unit whose output a unit's halo (K rows and one word around it,
    wrapping on the torus) reads is listed among its neighbours; the list is
    symmetric, so the unit that writes a buffer also waits for the readers of
    the previous pass (write-after-read on the double buffer).
These tests check both, and the unit shapes the kernel relies on, by brute
force over the plan that gol_plan_units reports from the library itself.
"""
import ctypes

import numpy as np
import pytest

gol = pytest.importorskip("paper_1209_4408_gb300.gol")

SUPPORTED_K = (1, 2, 3, 4, 5, 6, 7, 8, 16)
TILE_WORDS = 30
LANES = 32


@pytest.fixture(scope="module")
def lib():
    try:
        gol.load()
    except ImportError as e:
        pytest.skip(str(e))
    return gol


def cyclic_hits(a0, a1, b0, b1, n):
    """Whether [a0, a1) taken modulo n meets [b0, b1) (0 <= b0 < b1 <= n);
    a0, a1 are arrays."""
    a0 = np.asarray(a0)
    a1 = np.asarray(a1)
    hit = (a1 - a0) >= n
    for m in (-1, 0, 1):
        hit |= (a0 + m * n < b1) & (a1 + m * n > b0)
    return hit


def output_rects(u, words):
    """Output cells of a unit as (row0, row1, word0, word1) rectangles."""
    rects = []
    w0, w1 = (0, words) if u["mode"] == 0 else (u["w0"], u["w0"] + u["U"])
    for s in range(u["S"]):
        r0 = u["r0"] + s * u["H"]
        r1 = min(u["r0"] + (s + 1) * u["H"], u["r_end"])
        rects.append((r0, r1, w0, w1))
    return rects


def check_plan(rows, words, k, tile_rows, dense_limit=1 << 22):
    units = gol.gol_plan_units(rows, words, k, tile_rows)
    n = len(units)
    assert n >= 1
    cost = max(u["H"] for u in units) + 2 * k
    # shapes the kernel relies on
    for i, u in enumerate(units):
        assert 0 <= u["r0"] < u["r_end"] <= rows, u
        assert u["S"] >= 1 and u["H"] >= 1
        if u["mode"] == 0:
            assert words <= LANES and u["w0"] == 0 and u["U"] == words
            assert u["S"] * words <= LANES
            assert u["S"] == max(1, LANES // words) or u["S"] * u["H"] - u["H"] < u["r_end"] - u["r0"]
        else:
            assert u["mode"] == 1 and words > LANES and u["S"] == 1
            assert 1 <= u["U"] <= TILE_WORDS and u["U"] + 2 <= LANES
            assert 0 <= u["w0"] and u["w0"] + u["U"] <= words
        # every segment holds at least one row, none is past the block
        for r0, r1, _, _ in output_rects(u, words):
            assert u["r0"] <= r0 < r1 <= u["r_end"], u
        assert u["cost"] == cost
        assert 0 <= u["nnb"] <= 8
        assert len(set(u["nb"])) == u["nnb"] and i not in u["nb"]
        assert all(0 <= v < n for v in u["nb"])
    blocks = sorted({(u["r0"], u["r_end"]) for u in units})
    if len(blocks) > 1:
        assert min(b - a for a, b in blocks) >= k, "a halo must reach only the adjacent row blocks"
    # exact cover: row blocks partition the rows, tiles of a block partition the words
    assert blocks[0][0] == 0 and blocks[-1][1] == rows
    assert all(blocks[j][1] == blocks[j + 1][0] for j in range(len(blocks) - 1))
    if rows * words <= dense_limit:
        cover = np.zeros((rows, words), np.int32)
        for u in units:
            for r0, r1, w0, w1 in output_rects(u, words):
                cover[r0:r1, w0:w1] += 1
        assert (cover == 1).all()
    else:
        by_block = {}
        for u in units:
            by_block.setdefault(u["r0"], []).append((u["w0"], u["w0"] + u["U"]))
        for a, b in blocks:
            spans = sorted(by_block[a])
            assert spans[0][0] == 0 and spans[-1][1] == words
            assert all(spans[j][1] == spans[j + 1][0] for j in range(len(spans) - 1))
    # neighbours: symmetric, and a superset of the units the halo reads
    nbs = [set(u["nb"]) for u in units]
    for i in range(n):
        for v in nbs[i]:
            assert i in nbs[v], (i, v)
    if n <= 4096:
        R0 = np.array([u["r0"] for u in units])
        R1 = np.array([u["r_end"] for u in units])
        W0 = np.array([0 if u["mode"] == 0 else u["w0"] for u in units])
        W1 = np.array([words if u["mode"] == 0 else u["w0"] + u["U"] for u in units])
        for i, u in enumerate(units):
            # rows [r0 - K, r_end + K), words [w0 - 1, w0 + U + 1) (all words for full rows)
            rows_hit = cyclic_hits(R0 - k, R1 + k, u["r0"], u["r_end"], rows)
            if u["mode"] == 0:
                words_hit = np.ones(n, bool)
            else:
                words_hit = cyclic_hits(W0 - 1, W1 + 1, u["w0"], u["w0"] + u["U"], words)
            # units whose halo reads u's output are the units u must wait for
            readers = set(np.flatnonzero(rows_hit & words_hit).tolist()) - {i}
            assert readers <= nbs[i], (rows, words, k, tile_rows, i, sorted(readers - nbs[i]))
    return units


@pytest.mark.parametrize("rows,words,k,tile_rows", [
    (16384, 256, 8, 64),      # 16384^2 board, tuned
    (131072, 2048, 8, 512),   # 131072^2 board, tuned
    (2048, 32, 6, 128),       # widest board of the 4096-board batch
    (32, 1, 6, 128),          # narrowest
    (64, 1, 8, 128), (96, 2, 6, 128), (256, 3, 6, 128),
])
def test_workload_plans(lib, rows, words, k, tile_rows):
    check_plan(rows, words, k, tile_rows)


@pytest.mark.parametrize("k", [1, 2, 8, 16])
def test_boards_shorter_than_the_halo(lib, k):
    """Rows < K: one row block, whose halo wraps onto itself."""
    for rows in sorted({1, max(1, k // 2), max(1, k - 1)}):
        for words in (1, 5, 33, 61):
            units = check_plan(rows, words, k, 1)
            assert len({(u["r0"], u["r_end"]) for u in units}) == 1


def test_random_shapes(lib):
    rng = np.random.default_rng(1209)
    for _ in range(250):
        rows = int(np.exp(rng.uniform(0, np.log(5000))))
        words = int(np.exp(rng.uniform(0, np.log(300))))
        k = int(rng.choice(SUPPORTED_K))
        tile_rows = int(rng.choice([1, 3, 7, 16, 64, 128, 1000]))
        check_plan(max(1, rows), max(1, words), k, tile_rows)


def test_ragged_tile_edges(lib):
    """Words around multiples of the tile width and of the lane count."""
    for words in (29, 30, 31, 32, 33, 59, 60, 61, 62, 89, 90, 91):
        for k in (1, 6, 16):
            check_plan(3 * k + 1, words, k, k)


def test_plan_rejects_bad_arguments(lib):
    for args in ((0, 4, 6, 64), (4, 0, 6, 64), (4, 4, 9, 64), (4, 4, 6, 0), (4, 4, 0, 64),
                 ((1 << 31) - 1, (1 << 25) - 1, 1, 1)):          # more units than int32 ids
        with pytest.raises(gol.GolError):
            gol.gol_plan_units(*args)
    # a short buffer is an error, a NULL buffer only counts
    n = ctypes.c_size_t()
    l = gol.load()
    assert l.gol_plan_units(1024, 64, 6, 64, None, 0, ctypes.byref(n)) == 0 and n.value > 1
    buf = (ctypes.c_int32 * gol.UNIT_FIELDS)()
    assert l.gol_plan_units(1024, 64, 6, 64, buf, 1, ctypes.byref(n)) != 0
