"""Parity at full workload sizes, in the launch configuration bench.py times.

16384^2 board: the whole board against the oracle (its OpenMP row
decomposition, same arithmetic) after 1 and 10 generations, light-cone tiles
after 100, and the top-left 1024^2 crop run as its own torus in lockstep with
the oracle for 10000 generations.  4096-board batch: every board up to a fixed
oracle budget against the oracle, the largest boards against the same boards
stepped alone.  131072^2 board: the glider band against its known translation
and light-cone tiles against the oracle."""
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

    g.gol_set_option(g.GOL_OPT_GENS_PER_PASS, 0)
    g.gol_set_option(g.GOL_OPT_TILE_ROWS, 0)
    return g


def light_cone_tile(initial_region, t, T):
    """Oracle value of a T x T tile after t generations from the
    (T + 2t)^2 initial patch around it, run as its own torus."""
    return oracle.run_rows_omp(initial_region, t, THREADS)[t:t + T, t:t + T]


def check_tiles(b, cells_fn, t, T, starts):
    for (r0, c0) in starts:
        patch = cells_fn(r0 - t, c0 - t, T + 2 * t, T + 2 * t)
        want = light_cone_tile(patch, t, T)
        got = b.region(r0, c0, T, T)
        assert np.array_equal(got, want), "tile at (%d, %d) after %d generations" % (r0, c0, t)


def test_single_16k_board(gol):
    R = C = 16384
    W = C // 64
    seed = synth.SEED_SINGLE_16K
    words = synth.random_words(R, W, seed)
    cells = oracle.unpack_words(words)
    b = gol.Board(R, C)
    b.set_packed(words)
    b.step(1)
    x = oracle.run_rows_omp(cells, 1, THREADS)
    assert np.array_equal(oracle.unpack_words(b.get_packed()), x), "generation 1"
    b.step(9)
    x = oracle.run_rows_omp(x, 9, THREADS)
    assert np.array_equal(oracle.unpack_words(b.get_packed()), x), "generation 10"
    del x
    b.step(90)

    def cells_fn(r0, c0, nr, nc):
        return oracle.unpack_words(synth.random_words_region(W, seed, r0, nr, 0, W, R))[
            :, np.arange(c0, c0 + nc) % C]

    rng = np.random.default_rng(1)
    starts = [(0, 0), (R - 32, C - 32)] + [tuple(int(v) for v in rng.integers(0, R, 2)) for _ in range(6)]
    check_tiles(b, cells_fn, 100, 64, starts)
    assert b.generation() == 100
    b.close()


@pytest.mark.slow
def test_single_16k_crop_lockstep(gol):
    # the initial top-left 1024^2 crop as its own torus, 10000 generations,
    # compared with the oracle after every pass of the kernel
    R = C = 1024
    words = synth.random_words(16384, 256, synth.SEED_SINGLE_16K)[:R, :C // 64]
    x = oracle.unpack_words(words)
    b = gol.Board(R, C)
    b.set_packed(words)
    k, _ = gol.gol_tune_get(16384, 16384)
    g = 0
    while g < 10000:
        step = min(k, 10000 - g)
        b.step(step)
        x = oracle.run_rows_omp(x, step, THREADS)
        g += step
        assert np.array_equal(oracle.unpack_words(b.get_packed()), x), "crop after %d generations" % g
    b.close()


def test_batch_4096(gol):
    specs = synth.batch_specs(4096)
    boards, words = [], []
    for s in specs:
        w = synth.bernoulli_words(s.rows, s.cols, s.density, s.seed)
        b = gol.Board(s.rows, s.cols)
        b.set_packed(w)
        boards.append(b)
        words.append(w)
    gol.step_batch(boards, [s.gens for s in specs])
    # oracle on the cheapest boards first, up to a budget of cell updates
    order = sorted(range(len(specs)), key=lambda i: specs[i].cells * specs[i].gens)
    budget, used, checked = 6e9, 0, 0
    for i in order:
        cost = specs[i].cells * specs[i].gens
        if used + cost > budget:
            break
        want = oracle.run_rows_omp(oracle.unpack_words(words[i]), specs[i].gens, THREADS)
        assert np.array_equal(oracle.unpack_words(boards[i].get_packed()), want), "board %d" % i
        used += cost
        checked += 1
    assert checked >= 256
    # a seeded random sample of the large boards (both sides >= 1024: several
    # row blocks, multi-unit plans, the chain cap and the critical ring all at
    # work) against the oracle at their full generation counts
    big = [i for i, s in enumerate(specs) if s.rows >= 1024 and s.cols >= 1024]
    assert len(big) >= 100
    pick = [big[j] for j in np.random.default_rng(12345).permutation(len(big))[:8]]
    for i in pick:
        want = oracle.run_rows_omp(oracle.unpack_words(words[i]), specs[i].gens, THREADS)
        assert np.array_equal(oracle.unpack_words(boards[i].get_packed()), want), \
            "large board %d (%d x %d, %d generations)" % (i, specs[i].rows, specs[i].cols, specs[i].gens)
    # the most expensive boards: batch result equals the board stepped alone
    for i in order[-6:]:
        s = specs[i]
        alone = gol.Board(s.rows, s.cols)
        alone.set_packed(words[i])
        alone.step(s.gens)
        assert np.array_equal(alone.get_packed(), boards[i].get_packed()), "board %d alone vs batch" % i
        alone.close()
    for b in boards:
        b.close()


@pytest.mark.slow
def test_huge_131072_glider_band(gol):
    R = C = 131072
    W = C // 64
    seed = synth.SEED_HUGE_128K
    band = synth.GliderBand()
    words = synth.glider_band_words(R, W, seed, band)
    b = gol.Board(R, C)
    b.set_packed(words)
    lattice0 = band.glider_cells(0)

    def cells_fn(r0, c0, nr, nc):
        rr = np.arange(r0, r0 + nr) % R
        w0 = (c0 // 64) - 1
        nw = (nc + 63) // 64 + 2
        ww = words[np.ix_(rr, np.arange(w0, w0 + nw) % W)]
        full = oracle.unpack_words(ww)
        off = c0 - w0 * 64
        return np.ascontiguousarray(full[:, off:off + nc])

    g = 0
    for t in (100, 500, 1000):
        b.step(t - g)
        g = t
        lo, hi = band.b0 + t, band.b0 + band.band_rows - t
        region = b.region(lo, 0, hi - lo, C)
        rc = band.glider_cells(t)
        assert int(np.count_nonzero(region)) == len(rc), "band population after %d" % t
        assert region[rc[:, 0] - lo, rc[:, 1] % C].all(), "glider lattice after %d" % t
        del region
        if t == 100:
            rng = np.random.default_rng(2)
            starts = [(0, 0), (R - 40, C - 40)] + [tuple(int(v) for v in rng.integers(0, R, 2)) for _ in range(6)]
            check_tiles(b, cells_fn, 100, 64, starts)
        if t == 1000:
            check_tiles(b, cells_fn, 1000, 64, [(12345, 67890), (R - 32, 5)])
    assert len(lattice0) == 64 * 64 * 5
    b.close()
