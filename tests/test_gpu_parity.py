"""GPU parity: the CUDA path against the oracle, cell by cell (bit-exact).

Every expected value comes from ``oracle`` on inputs made by ``synth``; the
CUDA path is reached only through the C ABI (the ctypes binding)."""
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

    g.gol_set_option(g.GOL_OPT_GENS_PER_PASS, 0)
    g.gol_set_option(g.GOL_OPT_TILE_ROWS, 0)
    yield g
    g.gol_set_option(g.GOL_OPT_GENS_PER_PASS, 0)
    g.gol_set_option(g.GOL_OPT_TILE_ROWS, 0)


@pytest.fixture
def opts(gol):
    """Force generations per pass / tile rows, restoring the defaults."""
    def set_(k=0, rows=0):
        gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, k)
        gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, rows)
    yield set_
    set_(0, 0)


def run_gpu(gol, cells, gens, torus=True, layout=0):
    b = gol.Board(cells.shape[0], cells.shape[1], torus=torus, layout=layout)
    b.set(cells)
    b.step(gens)
    out = b.get()
    b.close()
    return out


def assert_same(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError("%s: %d cells differ, first at %s" % (what, len(bad), bad[:5].tolist()))


# ---------------------------------------------------------------------------
# byte-per-cell path
# ---------------------------------------------------------------------------
def test_bytes_256_every_generation(gol):
    # 256x256 torus, Bernoulli(0.3), 1000 generations, checked after each one
    R = C = 256
    cells = synth.bernoulli_board(R, C, 0.3, synth.SEED_BYTES_256)
    b = gol.Board(R, C, torus=True, layout=gol.GOL_LAYOUT_BYTES)
    b.set(cells)
    x = cells
    for g in range(1, 1001):
        b.step(1)
        x = oracle.step(x)
        assert_same(b.get(), x, "bytes 256x256 generation %d" % g)
    assert b.generation() == 1000
    assert b.population() == oracle.population(x)


@pytest.mark.parametrize("R,C", [(1, 1), (1, 3), (2, 2), (3, 3), (2, 5), (4, 3)])
@pytest.mark.parametrize("torus", [True, False])
def test_bytes_brute_force_tiny(gol, R, C, torus):
    b = gol.Board(R, C, torus=torus, layout=gol.GOL_LAYOUT_BYTES)
    for bits in range(1 << (R * C)):
        cells = np.array([(bits >> i) & 1 for i in range(R * C)], dtype=np.uint8).reshape(R, C)
        b.set(cells)
        b.step(1)
        assert_same(b.get(), oracle.step(cells, torus=torus), "bytes %dx%d state %d" % (R, C, bits))


@pytest.mark.parametrize("R,C", [(5, 7), (64, 100), (131, 67)])
def test_bytes_random_multi_gen(gol, R, C):
    cells = synth.bernoulli_board(R, C, 0.4, R * C)
    for torus in (True, False):
        assert_same(run_gpu(gol, cells, 17, torus, gol.GOL_LAYOUT_BYTES), oracle.run(cells, 17, torus),
                    "bytes %dx%d" % (R, C))


@pytest.mark.parametrize("cluster", [1, 0, 2, 8])
@pytest.mark.parametrize("R,C", [(1, 1), (2, 3), (9, 1), (7, 9), (16, 16), (33, 65), (100, 700), (960, 960),
                                 (1000, 1600), (1500, 1500), (2048, 2048), (3072, 3072)])
def test_bytes_cluster_and_per_generation_paths(gol, cluster, R, C):
    # boards whose cells fit, one bit each, in a cluster's shared memory
    # (two buffers of ceil(R / n) rows of ceil(C / 64) words per CTA, n <= 8:
    # 2048 x 2048 does) run all generations in one cluster launch; 3072 x
    # 3072 and option 0 take one launch per generation; options 2 and 8 force
    # that many CTAs where they fit (each strip at least one row); all match
    # the oracle, torus and bounded
    gol.gol_set_option(gol.GOL_OPT_BYTE_CLUSTER, cluster)
    try:
        cells = synth.bernoulli_board(R, C, 0.35, 7 * R + C)
        for torus in (True, False):
            b = gol.Board(R, C, torus=torus, layout=gol.GOL_LAYOUT_BYTES)
            b.set(cells)
            x = cells
            for g in (1, 2, 13):
                b.step(g)
                x = oracle.run(x, g, torus)
                assert_same(b.get(), x, "bytes %dx%d torus=%s cluster=%d" % (R, C, torus, cluster))
            assert b.generation() == 16
            b.close()
    finally:
        gol.gol_set_option(gol.GOL_OPT_BYTE_CLUSTER, 1)


# ---------------------------------------------------------------------------
# packed path: the rule at every bit position and across both wraps
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("R,C", [(8, 64), (64, 128), (5, 2112)])
def test_packed_all_512_neighbourhoods(gol, R, C):
    # each 3x3 neighbourhood on its own board, centred on a bit position in
    # {0, 1, 31, 32, 62, 63} of some word, on the first/last row and across
    # the left/right wrap; all boards stepped in one batch
    W = C // 64
    positions = []
    for bit in (0, 1, 31, 32, 62, 63):
        for word in sorted({0, W - 1, W // 2}):
            for row in sorted({0, R - 1, R // 2}):
                positions.append((row, 64 * word + bit))
    boards, starts = [], []
    for nb in range(512):
        pat = np.array([(nb >> i) & 1 for i in range(9)], dtype=np.uint8).reshape(3, 3)
        r, c = positions[nb % len(positions)]
        cells = np.zeros((R, C), dtype=np.uint8)
        for i in range(3):
            for j in range(3):
                cells[(r - 1 + i) % R, (c - 1 + j) % C] = pat[i, j]
        b = gol.Board(R, C, torus=True)
        b.set(cells)
        boards.append(b)
        starts.append(cells)
    gol.step_batch(boards, [1] * len(boards))
    for nb, (b, cells) in enumerate(zip(boards, starts)):
        assert_same(b.get(), oracle.step(cells), "neighbourhood %d on %dx%d" % (nb, R, C))
        b.close()


@pytest.mark.parametrize("torus", [True, False])
@pytest.mark.parametrize("R,C", [
    (1, 64), (2, 64), (3, 128), (7, 192), (64, 64), (100, 320), (257, 448), (33, 1024),
    (64, 1984), (50, 2048), (17, 2112), (40, 2880), (130, 4096), (9, 6400),
])
def test_packed_random_shapes(gol, opts, R, C, torus):
    cells = synth.bernoulli_board(R, C, 0.37, 1000 * R + C)
    try:
        for variant in (-1, 0, 2):
            gol.gol_set_option(gol.GOL_OPT_PIPELINE, variant)
            for k, rows in [(1, 0), (4, 3), (8, 0), (16, 64)]:
                opts(k, rows)
                for gens in (1, 5, 19):
                    assert_same(run_gpu(gol, cells, gens, torus), oracle.run(cells, gens, torus),
                                "%dx%d torus=%s K=%d rows=%d gens=%d variant=%d" % (R, C, torus, k, rows, gens,
                                                                                   variant))
    finally:
        gol.gol_set_option(gol.GOL_OPT_PIPELINE, -1)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8, 16])
@pytest.mark.parametrize("rows", [1, 8, 64, 1000])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_packed_result_independent_of_pass_and_tile(gol, opts, k, rows, variant):
    R, C, G = 192, 2240, 23
    cells = synth.bernoulli_board(R, C, 0.5, 4242)
    want = oracle.run(cells, G)
    opts(k, rows)
    gol.gol_set_option(gol.GOL_OPT_PIPELINE, variant)
    try:
        assert_same(run_gpu(gol, cells, G), want, "K=%d rows=%d variant=%d" % (k, rows, variant))
        # bounded board and a board narrow enough for several lane segments
        cells2 = synth.bernoulli_board(130, 320, 0.4, 77)
        assert_same(run_gpu(gol, cells2, G, torus=False), oracle.run(cells2, G, torus=False),
                    "bounded K=%d rows=%d variant=%d" % (k, rows, variant))
    finally:
        gol.gol_set_option(gol.GOL_OPT_PIPELINE, -1)


def test_packed_split_runs_compose(gol):
    cells = synth.bernoulli_board(160, 960, 0.45, 77)
    b = gol.Board(160, 960)
    b.set(cells)
    for g in (3, 0, 8, 1, 13):
        b.step(g)
    assert b.generation() == 25
    assert_same(b.get(), oracle.run(cells, 25), "split run")


@pytest.mark.parametrize("N", [64, 128, 1024])
def test_packed_glider_returns_after_4N(gol, N):
    cells = synth.pattern_board(N, N, "glider", N - 2, N - 3)
    b = gol.Board(N, N)
    b.set(cells)
    b.step(4 * N)
    assert_same(b.get(), cells, "glider on %dx%d" % (N, N))
    b.step(4)
    assert_same(b.get(), np.roll(cells, (1, 1), axis=(0, 1)), "glider moved")


def test_packed_still_lifes_and_blinker(gol):
    cells = np.zeros((64, 128), np.uint8)
    synth.place(cells, "block", 10, 62)       # straddles a word boundary
    synth.place(cells, "beehive", 63, 126)    # straddles both wraps
    synth.place(cells, "blinker", 30, 30)
    b = gol.Board(64, 128)
    b.set(cells)
    b.step(100)
    assert_same(b.get(), cells, "period-2 and still objects after 100 generations")
    b.step(1)
    assert not np.array_equal(b.get(), cells)


def test_closed_forms(gol):
    for R, C in [(3, 64), (64, 128), (40, 2112)]:
        assert not run_gpu(gol, np.ones((R, C), np.uint8), 1).any()
        r, c = np.indices((R + R % 2, C))
        chk = ((r + c) % 2 == 0).astype(np.uint8)
        assert not run_gpu(gol, chk, 1).any()
        assert not run_gpu(gol, np.zeros((R, C), np.uint8), 9).any()


def test_batch_equals_alone(gol):
    specs = synth.batch_specs(24, seed=5, side_hi=700, gen_lo=3, gen_hi=60)
    boards, cells = [], []
    for s in specs:
        c = synth.bernoulli_board(s.rows, s.cols, s.density, s.seed)
        b = gol.Board(s.rows, s.cols)
        b.set(c)
        boards.append(b)
        cells.append(c)
    gol.step_batch(boards, [s.gens for s in specs])
    for s, b, c in zip(specs, boards, cells):
        got = b.get()
        assert_same(got, oracle.run(c, s.gens), "batch board %d" % s.index)
        assert_same(got, run_gpu(gol, c, s.gens), "alone board %d" % s.index)
        assert b.generation() == s.gens


@pytest.mark.parametrize("critical", [0, 1, 500, 1000])
@pytest.mark.parametrize("k", [2, 6, 8])
def test_batch_queue_settings(gol, opts, critical, k):
    # the same results whatever share of the passes goes to the critical ring
    # (none, nearly all, half, only the longest chain), with tiles short
    # enough for many units per board and boards of one unit
    specs = synth.batch_specs(30, seed=31 + k, side_hi=900, gen_lo=4, gen_hi=90)
    gol.gol_set_option(gol.GOL_OPT_CRITICAL_PERMILLE, critical)
    opts(k, 16)
    try:
        boards, cells = [], []
        for s in specs:
            c = synth.bernoulli_board(s.rows, s.cols, s.density, s.seed)
            b = gol.Board(s.rows, s.cols)
            b.set(c)
            boards.append(b)
            cells.append(c)
        gol.step_batch(boards, [s.gens for s in specs])
        for s, b, c in zip(specs, boards, cells):
            assert_same(b.get(), oracle.run(c, s.gens), "critical %d K=%d board %d" % (critical, k, s.index))
            b.close()
    finally:
        gol.gol_set_option(gol.GOL_OPT_CRITICAL_PERMILLE, -1)


def test_batch_repeat_replays_graph(gol):
    import torch

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gol.gol_set_stream(stream)
        try:
            specs = synth.batch_specs(12, seed=8, side_hi=400, gen_lo=5, gen_hi=40)
            boards, cells = [], []
            for s in specs:
                c = synth.bernoulli_board(s.rows, s.cols, s.density, s.seed)
                b = gol.Board(s.rows, s.cols)
                b.set(c)
                boards.append(b)
                cells.append(c)
            for rep in range(4):          # first call launches, later ones replay a graph
                gol.step_batch(boards, [s.gens for s in specs])
            for s, b, c in zip(specs, boards, cells):
                assert_same(b.get(), oracle.run(c, 4 * s.gens), "graph replay board %d" % s.index)
        finally:
            gol.gol_set_stream(None)


@pytest.mark.parametrize("R,C", [(64, 1), (64, 65), (128, 3), (128, 100), (192, 1000), (640, 333), (1024, 2049)])
def test_packed_any_width_when_height_is_a_multiple_of_64(gol, opts, R, C):
    # a width that is not a multiple of 64 is packed, stored transposed
    # (whole words along the height); every way in and out that has a meaning
    # for it works, the packed word layout is refused
    cells = synth.bernoulli_board(R, C, 0.4, 17 * R + C)
    for torus in (True, False):
        b = gol.Board(R, C, torus=torus)
        assert gol.gol_info(b.handle)[3] == gol.GOL_LAYOUT_PACKED
        b.set(cells)
        assert_same(b.get(), cells, "round trip %dx%d" % (R, C))
        x = cells
        for g, k in ((1, 0), (5, 4), (21, 8)):
            opts(k, 0)
            b.step(g)
            x = oracle.run(x, g, torus)
            assert_same(b.get(), x, "%dx%d torus=%s after %d" % (R, C, torus, b.generation()))
        opts(0, 0)
        assert b.population() == oracle.population(x)
        reg = b.region(R - 3, C - 2, 7, min(C, 9))
        assert_same(reg, x[np.ix_(np.arange(R - 3, R + 4) % R, np.arange(C - 2, C - 2 + min(C, 9)) % C)],
                    "region %dx%d" % (R, C))
        with pytest.raises(gol.GolError):
            b.get_packed()
        b.close()
    # and in a batch beside other boards
    other = synth.bernoulli_board(64, 128, 0.4, 5)
    b1, b2 = gol.Board(R, C), gol.Board(64, 128)
    b1.set(cells)
    b2.set(other)
    gol.step_batch([b1, b2], [9, 4])
    assert_same(b1.get(), oracle.run(cells, 9), "batched %dx%d" % (R, C))
    assert_same(b2.get(), oracle.run(other, 4), "batched 64x128")


def test_mixed_layouts_and_edges_in_one_batch(gol):
    cases = [(50, 64, True, 0), (50, 64, False, 0), (30, 45, True, 0), (30, 45, False, 0), (70, 2176, False, 0)]
    boards, cells, gens = [], [], []
    for i, (R, C, t, lay) in enumerate(cases):
        c = synth.bernoulli_board(R, C, 0.4, 300 + i)
        b = gol.Board(R, C, torus=t, layout=lay)
        b.set(c)
        boards.append(b)
        cells.append(c)
        gens.append(7 + i)
    gol.step_batch(boards, gens)
    for (R, C, t, _), b, c, g in zip(cases, boards, cells, gens):
        assert_same(b.get(), oracle.run(c, g, t), "mixed %dx%d torus=%s" % (R, C, t))


def test_population_region_and_packed_io(gol):
    R, C = 96, 640
    cells = synth.bernoulli_board(R, C, 0.3, 11)
    b = gol.Board(R, C)
    b.set(cells)
    b.step(6)
    want = oracle.run(cells, 6)
    assert b.population() == oracle.population(want)
    reg = b.region(90, 600, 20, 70)               # straddles both wraps
    assert_same(reg, want[np.ix_(np.arange(90, 110) % R, np.arange(600, 670) % C)], "region")
    assert_same(oracle.unpack_words(b.get_packed()), want, "packed read")
    b2 = gol.Board(R, C)
    b2.set_packed(synth.pack_cells(want))
    assert_same(b2.get(), want, "packed write")


def test_torch_allocator_and_stream(gol):
    import torch

    stream = gol.use_torch_allocator()
    try:
        cells = synth.bernoulli_board(128, 256, 0.5, 3)
        assert_same(run_gpu(gol, cells, 12), oracle.run(cells, 12), "torch allocator")
        dev = torch.empty(128 * 4, dtype=torch.int64, device="cuda")
        b = gol.Board(128, 256)
        b.set(cells)
        b.step(3)
        gol.gol_get_packed_device(b.handle, dev.data_ptr(), dev.numel())
        stream.synchronize()
        got = dev.cpu().numpy().view(np.uint64).reshape(128, 4)
        assert_same(oracle.unpack_words(got), oracle.run(cells, 3), "device read")
    finally:
        gol.gol_set_allocator(None, None)
        gol.gol_set_stream(None)


def test_invalid_arguments(gol):
    # packed boards of any size (a partial last word when neither side is a
    # multiple of 64); an unknown layout is rejected
    with pytest.raises(gol.GolError) as e:
        gol.gol_create_ex(30, 100, True, 7)
    assert e.value.code == gol.GOL_EINVAL
    gol.gol_destroy(gol.gol_create_ex(30, 100, True, gol.GOL_LAYOUT_PACKED))
    gol.gol_destroy(gol.gol_create_ex(64, 100, True, gol.GOL_LAYOUT_PACKED))
    b = gol.Board(8, 64)
    bad = np.zeros((8, 64), np.uint8)
    bad[3, 5] = 2
    with pytest.raises(gol.GolError):
        b.set(bad)
    with pytest.raises(gol.GolError):
        b.step(-1)
    with pytest.raises(gol.GolError):
        gol.gol_step_batch([b.handle, b.handle], [1, 1])
    b2 = gol.Board(64, 64)
    with pytest.raises(gol.GolError):
        gol.gol_step_batch([b.handle, b2.handle, b.handle], [1, 1, 1])
    # a rejected call leaves the boards usable in the next batch
    gol.gol_step_batch([b2.handle, b.handle], [1, 2])
    gol.gol_step_batch([b.handle, b2.handle], [1, 1])
    gol.gol_sync(b.handle)
    assert gol.gol_generation(b.handle) == 3 and gol.gol_generation(b2.handle) == 2
    b2.close()
    with pytest.raises(gol.GolError):
        gol.gol_set(b.handle, np.zeros(10, np.uint8))
    for rows, cols in [(0, 64), (64, 0), (-1, 5)]:
        with pytest.raises(gol.GolError):
            gol.gol_create(rows, cols, True)


def test_bounded_wait_times_out_and_context_survives(gol):
    assert gol.gol_debug_unfilled_wait(200) == gol.GOL_ETIMEOUT
    cells = synth.bernoulli_board(64, 128, 0.5, 1)
    assert_same(run_gpu(gol, cells, 9), oracle.run(cells, 9), "after timeout")


def test_many_board_transfers(gol):
    specs = synth.batch_specs(9, seed=21, side_hi=600, gen_lo=2, gen_hi=30)
    boards = [gol.Board(s.rows, s.cols) for s in specs]
    cells = [synth.bernoulli_board(s.rows, s.cols, s.density, s.seed) for s in specs]
    flat = np.concatenate([synth.pack_cells(c).reshape(-1) for c in cells])
    hs = [b.handle for b in boards]
    gol.gol_set_packed_batch(hs, flat)
    gol.step_batch(boards, [s.gens for s in specs])
    out = np.empty_like(flat)
    gol.gol_get_packed_batch(hs, out)
    off = 0
    for s, b, c in zip(specs, boards, cells):
        n = s.rows * s.cols // 64
        want = oracle.run(c, s.gens)
        assert_same(oracle.unpack_words(out[off:off + n].reshape(s.rows, s.cols // 64)), want,
                    "batch transfer board %d" % s.index)
        assert_same(b.get(), want, "board %d" % s.index)
        assert b.generation() == s.gens
        off += n
    with pytest.raises(gol.GolError):
        gol.gol_set_packed_batch(hs, flat[:-1])
    with pytest.raises(gol.GolError):
        gol.gol_set_packed_batch(hs + hs[:1], np.concatenate([flat, flat[:specs[0].rows * specs[0].cols // 64]]))


@pytest.mark.parametrize("orient", [1, 2])
@pytest.mark.parametrize("zero_copy", [1, 0])
def test_many_board_transfers_pinned_and_pageable(gol, orient, zero_copy):
    # batch transfers through pinned host memory (read and written in place
    # unless zero copy is off) and through pageable memory (staged), on
    # boards whose 8 x 8-tile blocks are ragged in both directions
    import torch

    shapes = [(576, 704), (640, 1216), (128, 2176), (1088, 512), (64, 64), (192, 4032)]
    gol.gol_set_option(gol.GOL_OPT_ORIENTATION, orient)
    gol.gol_set_option(gol.GOL_OPT_ZERO_COPY, zero_copy)
    try:
        cells = [synth.bernoulli_board(R, C, 0.4, 1300 + i) for i, (R, C) in enumerate(shapes)]
        flat = np.concatenate([synth.pack_cells(c).reshape(-1) for c in cells])
        n = flat.size
        # a pinned buffer with the boards at an offset inside the allocation
        pin = torch.empty(n + 5, dtype=torch.int64, pin_memory=True)
        pinned = pin.numpy().view(np.uint64)[3:3 + n]
        for host_in in (pinned, flat.copy()):
            host_in[:] = flat
            boards = [gol.Board(R, C) for R, C in shapes]
            hs = [b.handle for b in boards]
            gol.gol_set_packed_batch(hs, host_in)
            out = np.zeros_like(flat)
            gol.gol_get_packed_batch(hs, out)
            np.testing.assert_array_equal(out, flat)
            gol.step_batch(boards, [9] * len(boards))
            pin_out = torch.zeros(n + 1, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)[1:]
            for host_out in (pin_out, np.zeros_like(flat)):
                gol.gol_get_packed_batch(hs, host_out)
                off = 0
                for (R, C), c in zip(shapes, cells):
                    k = R * C // 64
                    assert_same(oracle.unpack_words(host_out[off:off + k].reshape(R, C // 64)), oracle.run(c, 9),
                                "%dx%d orient %d zero copy %d" % (R, C, orient, zero_copy))
                    off += k
            for b in boards:
                b.close()
    finally:
        gol.gol_set_option(gol.GOL_OPT_ORIENTATION, 0)
        gol.gol_set_option(gol.GOL_OPT_ZERO_COPY, 1)


@pytest.mark.parametrize("orient", [1, 2])
def test_storage_orientation_all_io_paths(gol, orient):
    # the same results whether the library stores the board as is (1) or
    # transposed (2), through every way in and out of the device
    import torch

    gol.gol_set_option(gol.GOL_OPT_ORIENTATION, orient)
    try:
        shapes = [(64, 128), (128, 1216), (192, 64), (256, 2176), (64, 4096)]
        for i, (R, C) in enumerate(shapes):
            cells = synth.bernoulli_board(R, C, 0.45, 500 + i)
            want = oracle.run(cells, 13)
            for torus in (True, False):
                want_t = want if torus else oracle.run(cells, 13, torus=False)
                # bytes in, bytes out
                b = gol.Board(R, C, torus=torus)
                b.set(cells)
                b.step(13)
                assert_same(b.get(), want_t, "orient %d %dx%d torus=%s bytes" % (orient, R, C, torus))
                # packed out, region, population
                assert_same(oracle.unpack_words(b.get_packed()), want_t, "packed out")
                reg = b.region(R - 5, C - 7, 11, 19)
                assert_same(reg, want_t[np.ix_(np.arange(R - 5, R + 6) % R, np.arange(C - 7, C + 12) % C)], "region")
                assert b.population() == oracle.population(want_t)
                b.close()
            # packed in, device in and out
            b = gol.Board(R, C)
            b.set_packed(synth.pack_cells(cells))
            b.step(5)
            dev = torch.empty(R * C // 64, dtype=torch.int64, device="cuda")
            torch.cuda.synchronize()
            gol.gol_get_packed_device(b.handle, dev.data_ptr(), dev.numel())
            gol.gol_sync(b.handle)
            got = dev.cpu().numpy().view(np.uint64).reshape(R, C // 64)
            assert_same(oracle.unpack_words(got), oracle.run(cells, 5), "device out")
            gol.gol_set_packed_device(b.handle, dev.data_ptr(), dev.numel())
            b.step(8)
            assert_same(b.get(), want, "device in")
            b.close()
        # many-board transfers
        boards = [gol.Board(R, C) for R, C in shapes]
        cells = [synth.bernoulli_board(R, C, 0.3, 900 + i) for i, (R, C) in enumerate(shapes)]
        flat = np.concatenate([synth.pack_cells(c).reshape(-1) for c in cells])
        hs = [b.handle for b in boards]
        gol.gol_set_packed_batch(hs, flat)
        gol.step_batch(boards, [7] * len(boards))
        out = np.empty_like(flat)
        gol.gol_get_packed_batch(hs, out)
        off = 0
        for (R, C), c in zip(shapes, cells):
            n = R * C // 64
            assert_same(oracle.unpack_words(out[off:off + n].reshape(R, C // 64)), oracle.run(c, 7), "batch io")
            off += n
        for b in boards:
            b.close()
    finally:
        gol.gol_set_option(gol.GOL_OPT_ORIENTATION, 0)


@pytest.mark.parametrize("layout", [1, 2])
def test_population_trace(gol, layout):
    # populations after every 7 generations, the form of the paper's Table 1
    R, C = 96, 192
    cells = synth.bernoulli_board(R, C, 0.35, 61)
    b = gol.Board(R, C, layout=layout)
    b.set(cells)
    got = gol.gol_population_trace(b.handle, 7, 12)
    x, want = cells, []
    for _ in range(12):
        x = oracle.run(x, 7)
        want.append(oracle.population(x))
    assert [int(v) for v in got] == want
    assert b.generation() == 84
    assert_same(b.get(), x, "after the trace")
    b.close()


def test_bytes_graph_replay_on_torch_stream(gol):
    # long byte-board runs on a non-default stream replay a captured graph of
    # 64 generations; results match the oracle from either starting buffer
    import torch

    stream = torch.cuda.Stream()
    gol.gol_set_stream(stream)
    gol.gol_set_option(gol.GOL_OPT_BYTE_CLUSTER, 0)    # the per-generation launches
    try:
        cells = synth.bernoulli_board(100, 130, 0.35, 2)
        b = gol.Board(100, 130, layout=gol.GOL_LAYOUT_BYTES)
        b.set(cells)
        b.step(1)            # start the replays from the second buffer
        b.step(300)          # 4 replays + 44 single launches
        b.step(129)
        assert_same(b.get(), oracle.run(cells, 430), "byte graph replays")
        assert b.generation() == 430
        b.close()
    finally:
        gol.gol_set_option(gol.GOL_OPT_BYTE_CLUSTER, 1)
        gol.gol_set_stream(None)


@pytest.mark.parametrize("every", [1, 4, 7, 13])
def test_population_trace_batch(gol, every):
    # several boards traced at once: packed boards are counted inside the
    # step kernel at the end of the passes that end a sampling period (6
    # generations per pass: a period of 7 runs as passes of 4 + 3, 13 as
    # 5 + 4 + 4), byte boards sample by sample; torus and bounded, one unit
    # and many, full rows and word tiles, boards stored transposed
    shapes = [(96, 192, True), (640, 2176, True), (64, 3 * 64, True), (128, 100, True), (200, 64 * 40, False),
              (130, 256, False), (33, 47, True)]
    gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, 6)
    gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, 32)
    try:
        boards, cells = [], []
        for i, (R, C, torus) in enumerate(shapes):
            c = synth.bernoulli_board(R, C, 0.35, 500 + i)
            b = gol.Board(R, C, torus=torus)
            b.set(c)
            boards.append(b)
            cells.append(c)
        samples = 9
        got = gol.gol_population_trace_batch([b.handle for b in boards], every, samples)
        assert got.shape == (len(shapes), samples)
        for i, ((R, C, torus), c, b) in enumerate(zip(shapes, cells, boards)):
            x, want = c, []
            for _ in range(samples):
                x = oracle.run(x, every, torus)
                want.append(oracle.population(x))
            assert [int(v) for v in got[i]] == want, "board %d (%d x %d, torus %s)" % (i, R, C, torus)
            assert b.generation() == samples * every
            assert_same(b.get(), x, "board %d after the trace" % i)
        for b in boards:
            b.close()
    finally:
        gol.gol_set_option(gol.GOL_OPT_GENS_PER_PASS, 0)
        gol.gol_set_option(gol.GOL_OPT_TILE_ROWS, 0)


def test_population_trace_batch_rejects_bad_arguments(gol):
    b = gol.Board(64, 64)
    with pytest.raises(gol.GolError):
        gol.gol_population_trace_batch([b.handle, b.handle], 3, 2)
    with pytest.raises(gol.GolError):
        gol.gol_population_trace_batch([b.handle], 0, 2)
    b.close()


def test_two_batches_in_flight_on_two_streams(gol):
    # two sets of boards, each on its own stream, with uploads from pinned
    # memory and asynchronous downloads: each set's results equal the oracle,
    # whatever the other set's work in flight (staging buffers are returned
    # only after the work that used them)
    import torch

    gol.use_torch_allocator()              # staging buffers from PyTorch's caching allocator
    specs = synth.batch_specs(24, seed=31, side_hi=768, gen_lo=3, gen_hi=40)
    cells = [synth.bernoulli_board(s.rows, s.cols, s.density, s.seed) for s in specs]
    words = [synth.pack_cells(c) for c in cells]
    flat = np.concatenate([w.reshape(-1) for w in words])
    pin_in = torch.empty(flat.size, dtype=torch.int64, pin_memory=True)
    host_in = pin_in.numpy().view(np.uint64)
    host_in[:] = flat
    sets = [[gol.Board(s.rows, s.cols) for s in specs] for _ in range(2)]
    handles = [np.array([b.handle for b in bs], dtype=np.uint64) for bs in sets]
    outs = [torch.empty(flat.size, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64) for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    gens = np.array([s.gens for s in specs], dtype=np.int64)
    want = np.concatenate([synth.pack_cells(oracle.run(c, s.gens)).reshape(-1) for c, s in zip(cells, specs)])
    try:
        events = [None, None]
        for i in range(6):
            k = i % 2
            if events[k] is not None:
                events[k].synchronize()
                assert np.array_equal(outs[k], want), "set %d after step %d" % (k, i - 2)
                outs[k][:] = 0
            gol.gol_set_stream(streams[k])
            gol.gol_set_packed_batch(handles[k], host_in)
            gol.gol_step_batch(handles[k], gens)
            gol.gol_get_packed_batch_async(handles[k], outs[k])
            events[k] = torch.cuda.Event()
            events[k].record(streams[k])
        for k in range(2):
            events[k].synchronize()
            assert np.array_equal(outs[k], want), "set %d at the end" % k
    finally:
        gol.gol_set_stream(None)
        for bs in sets:
            for b in bs:
                b.close()
        gol.gol_set_allocator(None, None)
