"""Autotuner: the persisted table round-trips through the library (CPU), and a
tuning run on the GPU installs an entry under which results stay exact."""
import json

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1209_4408_gb300 import autotune, gol

    return autotune, gol


def test_table_save_and_load(mods, tmp_path):
    autotune, gol = mods
    entries = [{"rows": 512, "cols": 1024, "k": 5, "tile_rows": 48},
               {"rows": 4096, "cols": 8192, "k": 8, "tile_rows": 128}]
    path = str(tmp_path / "tune.json")
    autotune.save(entries, path)
    assert json.load(open(path))["entries"][0]["k"] == 5
    assert autotune.load(path) == 2
    assert gol.gol_tune_get(512, 1024) == (5, 48)
    assert gol.gol_tune_get(4096, 8192) == (8, 128)
    # a shape of another size class keeps the default
    k, rows = gol.gol_tune_get(64, 64)
    assert k >= 1 and rows >= 1
    with pytest.raises(gol.GolError):
        gol.gol_tune_set(64, 64, 9, 32)      # no kernel for 9 generations per pass
    gol.gol_tune_reset()
    assert gol.gol_tune_get(512, 1024) == gol.gol_tune_get(64, 64)


@pytest.mark.gpu
def test_tune_shape_on_gpu(mods):
    autotune, gol = mods
    res = autotune.tune_shape(256, 1024, gens=64, ks=(2, 4), tile_rows=(16, 64))
    assert gol.gol_tune_get(256, 1024) == (res["k"], res["tile_rows"])
    assert len(res["trials"]) == 4 and res["gcups"] > 0
    cells = synth.bernoulli_board(256, 1024, 0.4, 8)
    b = gol.Board(256, 1024)
    b.set(cells)
    b.step(33)
    assert np.array_equal(b.get(), oracle.run(cells, 33))
    b.close()
    gol.gol_tune_reset()


@pytest.mark.gpu
def test_tune_batch_on_gpu(mods):
    # per-class tuning on a small batch: the classes are ranked by work, the
    # entries found are installed, and the batch stays exact under them
    autotune, gol = mods
    import torch

    gol.gol_set_stream(torch.cuda.current_stream())
    specs = synth.batch_specs(40, seed=77, side_hi=512, gen_hi=200)
    boards, cells = [], []
    for s in specs:
        c = synth.bernoulli_board(s.rows, s.cols, s.density, s.seed)
        b = gol.Board(s.rows, s.cols)
        b.set(c)
        boards.append(b)
        cells.append(c)
    hs = [b.handle for b in boards]
    gens = [s.gens for s in specs]
    cls = autotune.batch_classes(hs, gens)
    assert abs(sum(c["share"] for c in cls) - 1.0) < 1e-9
    assert [c["work"] for c in cls] == sorted((c["work"] for c in cls), reverse=True)
    res = autotune.tune_batch(hs, gens, classes=2, tile_rows=(16, 64), ks=(4, 6), steps=1, warmup=1)
    assert len(res["entries"]) == 2 and res["after_s"] > 0
    for e in res["entries"]:
        assert gol.gol_tune_get(e["rows"], e["cols"]) == (e["k"], e["tile_rows"])
    for b, c in zip(boards, cells):           # restart from the initial cells under the tuned table
        b.set(c)
    gol.gol_step_batch(hs, gens)
    for b, c, s in zip(boards, cells, specs):
        assert np.array_equal(b.get(), oracle.run(c, s.gens)), (s.rows, s.cols, s.gens)
        b.close()
    gol.gol_tune_reset()
    autotune.load_shipped()
    gol.gol_set_stream(None)
