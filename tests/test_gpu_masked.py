"""Packed boards whose sides are not multiples of 64 (masked last word).

Such a board keeps each row as ceil(cols / 64) words, the last one holding
cols mod 64 columns; the step kernel carries the wrap across the partial word
(Section 2.2: left and right edges adjacent) or treats the outside as dead on
a bounded board.  Every result is compared cell by cell with the oracle."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def gol():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1209_4408_gb300 as g

    return g


def packed_board(gol, cells, torus):
    R, C = cells.shape
    b = gol.Board(R, C, torus=torus, layout=gol.GOL_LAYOUT_PACKED)
    b.set(cells)
    return b


@pytest.mark.parametrize("torus", [True, False])
@pytest.mark.parametrize("R", [63, 130, 3001])
@pytest.mark.parametrize("C", [65, 100, 2049])
def test_masked_widths_and_heights(gol, R, C, torus):
    cells = synth.bernoulli_board(R, C, 0.4, R * 7 + C)
    b = packed_board(gol, cells, torus)
    assert b.layout == gol.GOL_LAYOUT_PACKED
    x = cells
    for g in (1, 6, 13):                      # a pass of 1, one of 6, then 13 = two passes
        b.step(g)
        x = oracle.run_rows_omp(x, g, THREADS, torus)
        got = b.get()
        assert np.array_equal(got, x), "%d x %d torus=%s, %d differing cells" % (R, C, torus, int((got != x).sum()))
    assert b.population() == oracle.population(x)
    b.close()


@pytest.mark.parametrize("k,rows", [(4, 8), (6, 16), (8, 32)])
def test_masked_random_shapes_forced_plans(gol, k, rows):
    # random shapes with neither side a multiple of 64, several units per
    # board (short tiles), each generation count a mix of full and partial passes
    rng = np.random.default_rng(k * 100 + rows)
    gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, k)
    gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, rows)
    try:
        boards, want, gens = [], [], []
        for i in range(16):
            R, C = int(rng.integers(1, 300)), int(rng.integers(1, 300))
            if R % 64 == 0:
                R += 1
            if C % 64 == 0:
                C += 1
            torus = bool(i % 2)
            G = int(rng.integers(1, 40))
            cells = synth.bernoulli_board(R, C, 0.45, 900 + i)
            boards.append(packed_board(gol, cells, torus))
            want.append(oracle.run(cells, G, torus))
            gens.append(G)
        gol.step_batch(boards, gens)
        for b, w in zip(boards, want):
            assert np.array_equal(b.get(), w), (b.rows, b.cols, b.torus)
            b.close()
    finally:
        gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, 0)
        gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, 0)


@pytest.mark.parametrize("R,C", [(3, 3), (2, 5), (3, 4), (1, 7), (5, 2), (1, 1), (2, 1)])
def test_masked_every_state_of_tiny_boards(gol, R, C):
    # every state of a tiny board (tori count wrapped neighbours with
    # multiplicity), all in one batched launch, torus and bounded
    n = R * C
    states = ((np.arange(1 << n)[:, None] >> np.arange(n)) & 1).astype(np.uint8).reshape(-1, R, C)
    for torus in (True, False):
        boards = [packed_board(gol, s, torus) for s in states]
        gol.step_batch(boards, [2] * len(boards))
        for s, b in zip(states, boards):
            assert np.array_equal(b.get(), oracle.run(s, 2, torus)), (R, C, torus, s.tolist())
            b.close()


def test_masked_packed_io_region_and_transfers(gol):
    R, C = 200, 130                           # 3 words per row, 2 columns in the last one
    W = (C + 63) // 64
    cells = synth.bernoulli_board(R, C, 0.5, 11)
    words = np.zeros((R, W), dtype=np.uint64)
    words[:, :2] = synth.pack_cells(np.ascontiguousarray(cells[:, :128]))
    last = np.zeros((R, 64), np.uint8)
    last[:, :C - 128] = cells[:, 128:]
    words[:, 2] = synth.pack_cells(last)[:, 0]
    junk = words.copy()
    junk[:, 2] |= np.uint64(0xFFFF_FFFF_FFFF_FFFC)  # padding bits set on input are ignored
    b = gol.Board(R, C, layout=gol.GOL_LAYOUT_PACKED)
    b.set_packed(junk)
    assert np.array_equal(b.get(), cells)
    assert np.array_equal(b.get_packed(), words)          # padding comes back zero
    b.step(9)
    x = oracle.run(cells, 9)
    assert np.array_equal(b.region(R - 3, C - 4, 10, 12), x[np.ix_(np.arange(R - 3, R + 7) % R,
                                                                     np.arange(C - 4, C + 8) % C)])
    assert b.population() == oracle.population(x)
    # many-board transfers with masked boards among whole-word ones
    other = gol.Board(64, 128, layout=gol.GOL_LAYOUT_PACKED)
    ow = synth.random_words(64, 2, 5)
    flat = np.concatenate([junk.reshape(-1), ow.reshape(-1)])
    gol.gol_set_packed_batch([b.handle, other.handle], flat)
    out = np.zeros_like(flat)
    gol.gol_get_packed_batch([b.handle, other.handle], out)
    assert np.array_equal(out[:R * W].reshape(R, W), words)
    assert np.array_equal(out[R * W:].reshape(64, 2), ow)
    b.close()
    other.close()


def test_masked_population_trace(gol):
    shapes = [(100, 130, True), (77, 65, False), (130, 2049, True)]
    boards, cells = [], []
    for i, (R, C, torus) in enumerate(shapes):
        c = synth.bernoulli_board(R, C, 0.35, 40 + i)
        boards.append(packed_board(gol, c, torus))
        cells.append(c)
    got = gol.gol_population_trace_batch([b.handle for b in boards], 5, 6)
    for i, ((R, C, torus), c) in enumerate(zip(shapes, cells)):
        x, want = c, []
        for _ in range(6):
            x = oracle.run(x, 5, torus)
            want.append(oracle.population(x))
        assert [int(v) for v in got[i]] == want, shapes[i]
        assert np.array_equal(boards[i].get(), x)
        boards[i].close()


def test_auto_layout_of_large_odd_boards_is_packed(gol):
    # too large for one thread-block cluster's shared memory: packed, masked
    R, C = 5001, 3001
    b = gol.Board(R, C)
    assert b.layout == gol.GOL_LAYOUT_PACKED
    cells = synth.bernoulli_board(R, C, 0.3, 3)
    b.set(cells)
    b.step(3)
    assert np.array_equal(b.get(), oracle.run_rows_omp(cells, 3, THREADS))
    b.close()
    small = gol.Board(100, 130)                # fits a cluster: bytes
    assert small.layout == gol.GOL_LAYOUT_BYTES
    small.close()


@pytest.mark.parametrize("k", [4, 6, 8])
def test_masked_wide_boards_several_tiles(gol, k):
    # 71 and 96 words per row (three and four word tiles; on the torus tile 0
    # is rotated to hold the partial word and word 0), short row blocks
    gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, k)
    gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, 16)
    try:
        for (R, C, torus) in [(301, 64 * 70 + 13, True), (301, 64 * 70 + 13, False), (150, 64 * 95 + 50, True)]:
            cells = synth.bernoulli_board(R, C, 0.45, R * 3 + C + k)
            b = packed_board(gol, cells, torus)
            b.step(2 * k + 3)
            assert np.array_equal(b.get(), oracle.run_rows_omp(cells, 2 * k + 3, THREADS, torus)), (R, C, torus)
            b.close()
    finally:
        gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, 0)
        gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, 0)
