"""The allocation-free entry point (gol_step_packed_noalloc) against the
ordinary one (a board handle stepped with gol_step), on two calls in a row.

Callers that cannot allocate device memory while they step a board hand the
library their own board and spare buffer; the library keeps its scheduler
workspace in a static device array.  This file is collected last so that a
run stopping at its first failure has already run every other test; it also
passes on its own in a fresh process."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gol():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1209_4408_gb300 as g

    return g


def reference_after(gol, words, torus, gens):
    """The existing entry point: a handle created, set and stepped."""
    R, W = words.shape
    b = gol.Board(R, W * 64, torus=torus, layout=gol.GOL_LAYOUT_PACKED)
    b.set_packed(words)
    b.step(gens)
    out = b.get_packed()
    b.close()
    return out


@pytest.mark.parametrize("rows,cols,torus", [(200, 1024, True), (130, 2176, True), (97, 640, False),
                                             (3, 64, True)])
def test_noalloc_matches_handles_on_two_calls(gol, rows, cols, torus):
    import torch

    words = synth.bernoulli_words(rows, cols, 0.4, rows * 31 + cols)
    W = cols // 64
    stream = torch.cuda.Stream()
    board = torch.from_numpy(words.view(np.int64).copy()).cuda()
    spare = torch.empty_like(board)
    first, second = 37, 11
    with torch.cuda.stream(stream):
        gol.gol_step_packed_noalloc(board.data_ptr(), spare.data_ptr(), rows, cols, torus, first, stream)
        got1 = board.cpu().numpy().view(np.uint64).reshape(rows, W)
        gol.gol_step_packed_noalloc(board.data_ptr(), spare.data_ptr(), rows, cols, torus, second, stream)
        got2 = board.cpu().numpy().view(np.uint64).reshape(rows, W)
    want1 = reference_after(gol, words, torus, first)
    want2 = reference_after(gol, words, torus, first + second)
    assert np.array_equal(got1, want1), "first call"
    assert np.array_equal(got2, want2), "second call"
    if rows * cols <= 1 << 18:
        assert np.array_equal(oracle.unpack_words(got2),
                              oracle.run(oracle.unpack_words(words), first + second, torus))


def test_noalloc_rejects_sizes_beyond_the_workspace(gol):
    import torch

    board = torch.zeros(8, dtype=torch.int64, device="cuda")
    spare = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(gol.GolError) as e:
        gol.gol_step_packed_noalloc(board.data_ptr(), spare.data_ptr(), 1, 64 * 30 * 4096 + 64, True, 1)
    assert e.value.code == gol.GOL_EINVAL
    with pytest.raises(gol.GolError):
        gol.gol_step_packed_noalloc(board.data_ptr(), board.data_ptr(), 1, 64, True, 1)


def light_cone_ok(words, got_words, gens, starts, T=64):
    """Each T x T tile of the result equals the oracle run on the (T + 2 gens)^2
    initial patch around it as its own torus (a cell at generation t depends
    only on initial cells within Chebyshev distance t)."""
    import os

    R, W = words.shape
    C = W * 64
    got = oracle.unpack_words(got_words)
    init = oracle.unpack_words(words)
    for r0, c0 in starts:
        rr = np.arange(r0 - gens, r0 + T + gens) % R
        cc = np.arange(c0 - gens, c0 + T + gens) % C
        want = oracle.run_rows_omp(init[np.ix_(rr, cc)], gens, max(1, os.cpu_count() or 1))[gens:gens + T,
                                                                                            gens:gens + T]
        tile = got[np.ix_(np.arange(r0, r0 + T) % R, np.arange(c0, c0 + T) % C)]
        if not np.array_equal(tile, want):
            return False
    return True


def noalloc_two_calls(gol, words, torus, first, second):
    import torch

    rows, W = words.shape
    stream = torch.cuda.Stream()
    board = torch.from_numpy(words.view(np.int64).copy()).cuda()
    spare = torch.empty_like(board)
    with torch.cuda.stream(stream):
        gol.gol_step_packed_noalloc(board.data_ptr(), spare.data_ptr(), rows, W * 64, torus, first, stream)
        got1 = board.cpu().numpy().view(np.uint64).reshape(rows, W)
        gol.gol_step_packed_noalloc(board.data_ptr(), spare.data_ptr(), rows, W * 64, torus, second, stream)
        got2 = board.cpu().numpy().view(np.uint64).reshape(rows, W)
    return got1, got2


def test_noalloc_several_launches_with_odd_pass_counts(gol):
    # 16000 x 3840 cells: 60 words per row = two 30-word tiles; with 8-row
    # tiles the board has 2000 row blocks x 2 tiles = 4000 units, so one
    # launch holds floor(2^18 / 4000) = 65 passes.  At 6 generations per pass
    # the first call (468 generations = 78 passes) runs launches of 65 and 13
    # passes, the second (785 = 65 + 65 + 1 passes, the last one 5
    # generations long) three launches, ending on the spare buffer.
    rows, cols = 16000, 3840
    words = synth.bernoulli_words(rows, cols, 0.35, 4242)
    assert len(gol.gol_plan_units(rows, cols // 64, 6, 8)) == 4000
    gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, 6)
    gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, 8)
    try:
        first, second = 468, 785
        got1, got2 = noalloc_two_calls(gol, words, True, first, second)
    finally:
        gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, 0)
        gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, 0)
    assert np.array_equal(got1, reference_after(gol, words, True, first)), "first call"
    assert np.array_equal(got2, reference_after(gol, words, True, first + second)), "second call"
    assert light_cone_ok(words, got1, first, [(0, 0), (rows - 32, cols - 32), (7919, 1000)])


def test_noalloc_board_needing_taller_units(gol):
    # 4-row tiles would give the same board 5332 units, more than the
    # workspace holds: the call must take taller units (4000 of them here).
    rows, cols = 16000, 3840
    assert len(gol.gol_plan_units(rows, cols // 64, 6, 4)) > 4096
    words = synth.bernoulli_words(rows, cols, 0.5, 77)
    gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, 6)
    gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, 4)
    try:
        got1, got2 = noalloc_two_calls(gol, words, False, 100, 31)
    finally:
        gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, 0)
        gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, 0)
    assert np.array_equal(got1, reference_after(gol, words, False, 100)), "first call"
    assert np.array_equal(got2, reference_after(gol, words, False, 131)), "second call"


@pytest.mark.parametrize("rows,cols", [(128, 1920), (640, 64 * 17)])
def test_noalloc_rows_multiple_of_64(gol, rows, cols):
    # boards whose height is a multiple of 64 may be stored transposed by the
    # handle path: the comparison then crosses the two storage layouts
    words = synth.bernoulli_words(rows, cols, 0.3, rows + cols)
    got1, got2 = noalloc_two_calls(gol, words, True, 50, 23)
    assert np.array_equal(got1, reference_after(gol, words, True, 50)), "first call"
    assert np.array_equal(got2, reference_after(gol, words, True, 73)), "second call"
    assert np.array_equal(oracle.unpack_words(got2), oracle.run(oracle.unpack_words(words), 73, True))
