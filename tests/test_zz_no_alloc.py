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
