"""Pins of the oracle to what the paper and the mathematics fix.

None of these compares the oracle with itself: each expected value comes
from a different formulation (rule sets, a set-of-live-cells simulator, a
numpy roll-sum), from closed forms, from hand-derived pattern phases
(tests/golden/patterns.txt), or from invariants of the rule (symmetry,
translation, composition, the light cone).
"""
import itertools
from collections import Counter

import numpy as np
import pytest

import oracle
import synth
from conftest import golden_patterns, read_golden

# B3/S23 as rule sets (Section 1: birth with exactly 3, survival with 2 or 3).
BIRTH = {3}
SURVIVE = {2, 3}


# ---------------------------------------------------------------------------
# Independent formulations used as expected values
# ---------------------------------------------------------------------------
def life_by_live_set(live, R, C, torus=True):
    """Set-of-live-cells simulator: every live cell adds one to each of its
    eight neighbours (with multiplicity on tiny tori); cells are then kept or
    born from the rule sets."""
    counts = Counter()
    for (r, c) in live:
        for dr in (-1, 0, 1):
            for dc in (-1, 0, 1):
                if dr == 0 and dc == 0:
                    continue
                rr, cc = r + dr, c + dc
                if torus:
                    counts[(rr % R, cc % C)] += 1
                elif 0 <= rr < R and 0 <= cc < C:
                    counts[(rr, cc)] += 1
    nxt = set()
    for cell, n in counts.items():
        if (cell in live and n in SURVIVE) or (cell not in live and n in BIRTH):
            nxt.add(cell)
    return nxt


def life_by_roll(states):
    """numpy roll-sum over a stack of tori: states[N, R, C] -> next states."""
    n = np.zeros(states.shape, dtype=np.int32)
    for dr in (-1, 0, 1):
        for dc in (-1, 0, 1):
            if dr or dc:
                n += np.roll(states, shift=(dr, dc), axis=(1, 2))
    alive = states.astype(bool)
    return ((~alive & (n == 3)) | (alive & ((n == 2) | (n == 3)))).astype(np.uint8)


def to_set(cells):
    return {(int(r), int(c)) for r, c in zip(*np.nonzero(cells))}


def from_set(live, R, C):
    b = np.zeros((R, C), dtype=np.uint8)
    for r, c in live:
        b[r, c] = 1
    return b


# ---------------------------------------------------------------------------
# The four transitions over all 512 neighbourhoods
# ---------------------------------------------------------------------------
def all_neighbourhoods():
    for bits in range(512):
        yield np.array([(bits >> i) & 1 for i in range(9)], dtype=np.uint8).reshape(3, 3)


@pytest.mark.parametrize("R,C,r0,c0,torus", [
    (3, 3, 0, 0, True),     # the 3x3 torus: centre's 8 neighbours are the other 8 cells once each
    (5, 5, 1, 1, False),    # interior of a bounded board
    (5, 7, 4, 6, True),     # neighbourhood straddling both wraps
    (6, 5, 0, 3, True),
])
def test_rule_all_512_neighbourhoods(R, C, r0, c0, torus):
    for nb in all_neighbourhoods():
        board = np.zeros((R, C), dtype=np.uint8)
        for i in range(3):
            for j in range(3):
                board[(r0 + i) % R, (c0 + j) % C] = nb[i, j]
        out = oracle.step(board, torus=torus)
        centre = ((r0 + 1) % R, (c0 + 1) % C)
        n = int(nb.sum()) - int(nb[1, 1])
        alive = bool(nb[1, 1])
        expect = (n in SURVIVE) if alive else (n in BIRTH)
        assert out[centre] == int(expect), (nb, n, alive)


def test_each_transition_named_in_section_1():
    # one witness per transition, on a 3x3 torus (centre's neighbours = the other 8 cells)
    def centre_after(alive, n):
        nb = np.zeros(9, dtype=np.uint8)
        order = [0, 1, 2, 3, 5, 6, 7, 8]
        nb[order[:n]] = 1
        nb[4] = alive
        return int(oracle.step(nb.reshape(3, 3))[1, 1])
    for n in range(9):
        # 1: under-population, 2: lives on, 3: overcrowding
        assert centre_after(1, n) == (1 if n in (2, 3) else 0)
        # 4: reproduction; any other count leaves a dead cell dead
        assert centre_after(0, n) == (1 if n == 3 else 0)


# ---------------------------------------------------------------------------
# Still lifes, oscillators, gliders (phases from tests/golden/patterns.txt)
# ---------------------------------------------------------------------------
PAT = golden_patterns()


def pattern_at(name, phase, R, C, r, c):
    b = np.zeros((R, C), dtype=np.uint8)
    for dr, dc in PAT[(name, phase)]:
        b[(r + dr) % R, (c + dc) % C] = 1
    return b


def test_golden_phase0_matches_synth_patterns():
    for name in ("glider", "blinker", "block", "beehive"):
        assert PAT[(name, 0)] == set(synth.PATTERNS[name])


@pytest.mark.parametrize("torus", [True, False])
@pytest.mark.parametrize("name,period", [("block", 1), ("beehive", 1), ("blinker", 2)])
def test_still_lifes_and_blinker(name, period, torus):
    # the hand-derived phases: phase 1 of a still life is phase 0, phase 2 of
    # the blinker is phase 0, phase 1 of the blinker is not
    assert (PAT[(name, 1)] == PAT[(name, 0)]) == (period == 1)
    if period == 2:
        assert PAT[("blinker", 2)] == PAT[("blinker", 0)]
    b0 = pattern_at(name, 0, 16, 16, 5, 6)
    for g in range(1, 5):
        expect = pattern_at(name, 1 if (period == 2 and g % 2) else 0, 16, 16, 5, 6)
        assert np.array_equal(oracle.run(b0, g, torus=torus), expect), (name, g)
    assert np.array_equal(oracle.run(b0, 100, torus=torus), b0)
    assert np.array_equal(oracle.run(b0, 101, torus=torus), pattern_at(name, period - 1, 16, 16, 5, 6))


def test_glider_phases():
    b = pattern_at("glider", 0, 12, 12, 3, 4)
    for g in range(1, 5):
        b = oracle.step(b)
        assert np.array_equal(b, pattern_at("glider", g, 12, 12, 3, 4)), g
    # phase 4 is phase 0 moved one row down and one column right
    assert np.array_equal(b, pattern_at("glider", 0, 12, 12, 4, 5))


@pytest.mark.parametrize("N", [8, 17, 64])
def test_glider_returns_after_4N_on_NxN_torus(N):
    b0 = pattern_at("glider", 0, N, N, N - 2, N - 3)   # starts straddling both wraps
    assert np.array_equal(oracle.run(b0, 4 * N), b0)
    for g in (4, 4 * N - 4):
        assert not np.array_equal(oracle.run(b0, g), b0)
    # after 4t generations it is the start translated by (t, t)
    t = 5
    assert np.array_equal(oracle.run(b0, 4 * t), np.roll(b0, (t, t), axis=(0, 1)))


def test_glider_dies_at_bounded_corner():
    # bounded board: the glider runs into the corner and becomes a block (still life)
    b0 = pattern_at("glider", 0, 8, 8, 0, 0)
    b = oracle.run(b0, 40, torus=False)
    assert np.array_equal(oracle.step(b, torus=False), b)
    assert oracle.population(b) == 4


# ---------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("R,C", [(1, 1), (1, 5), (3, 3), (7, 64), (64, 3)])
def test_all_dead_stays_dead(R, C):
    z = np.zeros((R, C), dtype=np.uint8)
    for torus in (True, False):
        assert not oracle.run(z, 7, torus=torus).any()


@pytest.mark.parametrize("R,C", [(3, 3), (4, 9), (64, 64), (5, 130)])
def test_all_live_torus_dies(R, C):
    # every cell has 8 live neighbours
    assert not oracle.step(np.ones((R, C), dtype=np.uint8)).any()


def test_all_live_bounded_board():
    # bounded: corners have 3 neighbours (survive), edges 5, interior 8 (die)
    b = oracle.step(np.ones((6, 7), dtype=np.uint8), torus=False)
    expect = np.zeros((6, 7), dtype=np.uint8)
    expect[0, 0] = expect[0, -1] = expect[-1, 0] = expect[-1, -1] = 1
    assert np.array_equal(b, expect)


@pytest.mark.parametrize("R,C", [(2, 2), (4, 6), (64, 128), (10, 64)])
def test_even_checkerboard_torus_dies(R, C):
    # live cells see 4 live diagonals, dead cells 4 live orthogonals
    r, c = np.indices((R, C))
    chk = ((r + c) % 2 == 0).astype(np.uint8)
    assert not oracle.step(chk).any()


def test_one_by_one_torus():
    # a live cell is its own neighbour eight times: n = 8, it dies
    assert oracle.step(np.ones((1, 1), np.uint8))[0, 0] == 0
    assert oracle.step(np.zeros((1, 1), np.uint8))[0, 0] == 0


@pytest.mark.parametrize("C", [1, 2, 3, 5, 9])
def test_single_row_torus_closed_form(C):
    # R = 1: offsets (+-1, 0) name the cell itself, (+-1, +-1) and (0, +-1) its
    # row neighbours, so n(c) = 2 x[c] + 3 x[c-1] + 3 x[c+1].
    for bits in range(1 << C):
        x = np.array([(bits >> i) & 1 for i in range(C)], dtype=np.uint8)
        n = 2 * x + 3 * np.roll(x, 1) + 3 * np.roll(x, -1)
        expect = np.where(x == 1, np.isin(n, [2, 3]), n == 3).astype(np.uint8)
        assert np.array_equal(oracle.step(x[None, :])[0], expect), (C, bits)


# ---------------------------------------------------------------------------
# Brute force on tiny boards
# ---------------------------------------------------------------------------
TINY = [(1, 1), (1, 2), (2, 1), (1, 4), (2, 2), (2, 3), (3, 2), (1, 8), (3, 3), (2, 5), (3, 4), (4, 3)]


@pytest.mark.parametrize("R,C", TINY)
@pytest.mark.parametrize("torus", [True, False])
def test_brute_force_vs_live_set(R, C, torus):
    for bits in range(1 << (R * C)):
        cells = np.array([(bits >> i) & 1 for i in range(R * C)], dtype=np.uint8).reshape(R, C)
        expect = from_set(life_by_live_set(to_set(cells), R, C, torus), R, C)
        assert np.array_equal(oracle.step(cells, torus=torus), expect), (R, C, bits)


@pytest.mark.parametrize("R,C", [(4, 4), (2, 8), (8, 2)])
def test_brute_force_vs_roll(R, C):
    n = 1 << (R * C)
    idx = np.arange(n, dtype=np.uint32)
    states = ((idx[:, None] >> np.arange(R * C, dtype=np.uint32)[None, :]) & 1).astype(np.uint8)
    states = states.reshape(n, R, C)
    expect = life_by_roll(states)
    lib = oracle._load()
    out = np.empty((R, C), dtype=np.uint8)
    for i in range(n):
        s = np.ascontiguousarray(states[i])
        assert lib.oracle_step(R, C, 1, s.ctypes.data, out.ctypes.data) == 0
        if not np.array_equal(out, expect[i]):
            raise AssertionError((R, C, i))


# ---------------------------------------------------------------------------
# Invariants on random boards
# ---------------------------------------------------------------------------
def rand_board(R, C, p=0.35, seed=7):
    return synth.bernoulli_board(R, C, p, seed)


@pytest.mark.parametrize("R,C", [(17, 23), (64, 128), (9, 200)])
def test_random_boards_vs_roll(R, C):
    b = rand_board(R, C)
    x = b
    for g in range(12):
        x_next = life_by_roll(x[None])[0]
        assert np.array_equal(oracle.step(x), x_next), g
        x = x_next


def test_translation_equivariance():
    b = rand_board(40, 130)
    out = oracle.run(b, 6)
    for a, c in [(1, 1), (0, 63), (5, 64), (39, 129), (13, 65)]:
        assert np.array_equal(oracle.run(np.roll(b, (a, c), axis=(0, 1)), 6),
                              np.roll(out, (a, c), axis=(0, 1)))


def test_d4_symmetry_square_torus():
    b = rand_board(48, 48, seed=11)
    out = oracle.run(b, 5)
    for f in (np.transpose, np.flipud, np.fliplr, lambda a: np.rot90(a, 1), lambda a: np.rot90(a, 2)):
        assert np.array_equal(oracle.run(np.ascontiguousarray(f(b)), 5), f(out))


def test_composition():
    b = rand_board(33, 70, seed=3)
    for g1, g2 in [(0, 5), (3, 4), (7, 0), (1, 1)]:
        assert np.array_equal(oracle.run(oracle.run(b, g1), g2), oracle.run(b, g1 + g2))


@pytest.mark.parametrize("torus", [True, False])
def test_decompositions_equal_serial(torus):
    b = rand_board(61, 47, seed=5)
    ref = oracle.run(b, 9, torus=torus)
    for th in (1, 2, 3, 4, 8):
        assert np.array_equal(oracle.run_rows_omp(b, 9, th, torus=torus), ref)
        assert np.array_equal(oracle.run_cols_omp(b, 9, th, torus=torus), ref)
    for m, n in [(2, 2), (3, 2), (1, 4)]:
        assert np.array_equal(oracle.run_blocks_omp(b, 9, m, n, torus=torus), ref)


def test_r_pentomino_stabilises_at_1103_with_116_cells():
    """A known property of B3/S23, independent of the paper: the R-pentomino
    is a methuselah whose population settles at generation 1103 at 116 cells
    (still lifes, blinkers and six escaping gliders), 118 the generation
    before.  On a 768 x 768 torus nothing wraps into the debris by then."""
    import os

    N = 768
    b = np.zeros((N, N), np.uint8)
    for dr, dc in [(0, 1), (0, 2), (1, 0), (1, 1), (2, 1)]:       # .XX / XX. / .X.
        b[N // 2 + dr, N // 2 + dc] = 1
    threads = max(1, os.cpu_count() or 1)
    x = oracle.run_rows_omp(b, 1102, threads)
    assert int(x.sum()) == 118
    for _ in range(3):                                              # generations 1103 .. 1105
        x = oracle.run_rows_omp(x, 1, threads)
        assert int(x.sum()) == 116


def _place_rows(N, rows, r0, c0):
    b = np.zeros((N, N), np.uint8)
    for r, line in enumerate(rows):
        for c, ch in enumerate(line):
            b[r0 + r, c0 + c] = ch == "O"
    return b


def test_diehard_vanishes_at_generation_130():
    """Known property of B3/S23: the seven-cell Diehard dies out after
    exactly 130 generations."""
    x = _place_rows(128, ["......O.", "OO......", ".O...OOO"], 60, 60)
    x = oracle.run(x, 129)
    assert int(x.sum()) > 0
    assert int(oracle.run(x, 1).sum()) == 0


def test_lightweight_spaceship_moves_two_cells_per_four_generations():
    """Known property of B3/S23: the lightweight spaceship (period 4, nine
    cells) travels at c/2; on an N-wide torus it is home after 2N
    generations."""
    N = 40
    b = _place_rows(N, [".O..O", "O....", "O...O", "OOOO."], 18, 20)
    assert np.array_equal(oracle.run(b, 4), np.roll(b, -2, axis=1))
    assert np.array_equal(oracle.run(b, 2 * N), b)


def test_light_cone():
    # cell (r, c) after t generations depends only on initial cells within
    # Chebyshev distance t: a T x T tile equals the centre of the run on the
    # (T + 2t)-patch around it treated as its own torus.
    R, C, T = 96, 160, 16
    b = rand_board(R, C, seed=9)
    for t in (1, 4, 10):
        full = oracle.run(b, t)
        for (r0, c0) in [(0, 0), (40, 70), (90, 150)]:
            rr = np.arange(r0 - t, r0 + T + t) % R
            cc = np.arange(c0 - t, c0 + T + t) % C
            patch = b[np.ix_(rr, cc)]
            tile = oracle.run(patch, t)[t:t + T, t:t + T]
            want = full[np.ix_(np.arange(r0, r0 + T) % R, np.arange(c0, c0 + T) % C)]
            assert np.array_equal(tile, want), (t, r0, c0)


def test_population():
    b = rand_board(50, 70)
    assert oracle.population(b) == int(b.sum())
    assert oracle.population(np.zeros((3, 0), np.uint8)) == 0


def test_empty_boards():
    for shape in [(0, 0), (0, 5), (5, 0)]:
        z = np.zeros(shape, dtype=np.uint8)
        assert oracle.run(z, 3).shape == shape
        assert oracle.step(z).shape == shape


def test_invalid_arguments():
    lib = oracle._load()
    assert lib.oracle_step(-1, 3, 1, None, None) != 0
    b = np.zeros((2, 2), np.uint8)
    assert lib.oracle_run(2, 2, 1, -1, b.ctypes.data, b.ctypes.data) != 0


# ---------------------------------------------------------------------------
# Generators and the packed layout
# ---------------------------------------------------------------------------
def test_splitmix64_reference_outputs():
    rows = [ln.split() for ln in read_golden("splitmix64.txt")]
    state = 0
    for i, hx in rows:
        assert synth.sm64_int(state) == int(hx, 16)
        assert int(synth.sm64(np.uint64(state))) == int(hx, 16)
        state = (state + 0x9E3779B97F4A7C15) % (1 << 64)


def test_sm64_vector_matches_scalar():
    xs = [0, 1, 2 ** 63, 2 ** 64 - 1, 123456789]
    v = synth.sm64(np.array(xs, dtype=np.uint64))
    assert [int(a) for a in v] == [synth.sm64_int(x) for x in xs]


def test_bernoulli_board_definition_and_region():
    R, C, p, s = 9, 130, 0.3, 42
    b = synth.bernoulli_board(R, C, p, s)
    for (r, c) in [(0, 0), (3, 77), (8, 129)]:
        u = (synth.sm64_int(s + r * C + c) >> 11) * 2.0 ** -53
        assert b[r, c] == int(u < p)
    assert np.array_equal(synth.bernoulli_region(R, C, p, s, 7, 120, 5, 20),
                          b[np.ix_(np.arange(7, 12) % R, np.arange(120, 140) % C)])
    assert abs(synth.bernoulli_board(256, 256, 0.3, 1).mean() - 0.3) < 0.01


def test_random_words_definition_and_region():
    w = synth.random_words(5, 3, 99)
    assert int(w[4, 2]) == synth.sm64_int(99 + 4 * 3 + 2)
    assert np.array_equal(synth.random_words_region(3, 99, 3, 4, 2, 2, 5),
                          w[np.ix_([3, 4, 0, 1], [2, 0])])


def test_packed_bit_order():
    # bit j of word k is column 64k + j, checked one cell at a time
    for c in (0, 1, 31, 32, 63, 64, 65, 127):
        cells = np.zeros((2, 128), np.uint8)
        cells[1, c] = 1
        w = synth.pack_cells(cells)
        assert int(w[1, c // 64]) == 1 << (c % 64) and int(w[0].sum()) == 0
        assert np.array_equal(oracle.unpack_words(w), cells)
    b = rand_board(7, 192)
    assert np.array_equal(oracle.unpack_words(synth.pack_cells(b)), b)


def test_batch_specs_shapes():
    specs = synth.batch_specs(4096)
    rows = np.array([s.rows for s in specs])
    cols = np.array([s.cols for s in specs])
    gens = np.array([s.gens for s in specs])
    assert rows.min() >= 64 and rows.max() <= 2048 and (rows % 64 == 0).all()
    assert cols.min() >= 64 and cols.max() <= 2048 and (cols % 64 == 0).all()
    assert gens.min() >= 100 and gens.max() <= 5000
    assert synth.batch_specs(4096)[17] == specs[17]          # deterministic
    assert len({s.seed for s in specs}) == len(specs)        # distinct board seeds


def test_request_stream_recipe():
    """Poisson arrivals (exponential gaps of mean 1/rate), sides multiples of
    64 in [64, 8192], densities in [0.1, 0.6], generations in [10, 1e5]."""
    n, rate = 4000, 650.0
    reqs = synth.request_stream(n, rate)
    t = np.array([r.arrival_s for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    # the mean of n exponential gaps is within 5 standard errors of 1/rate
    assert abs(gaps.mean() - 1 / rate) < 5 * (1 / rate) / np.sqrt(n)
    # exponential: the gaps' standard deviation equals their mean
    assert abs(gaps.std() / gaps.mean() - 1) < 0.1
    sides = np.array([(r.rows, r.cols) for r in reqs])
    assert (sides % 64 == 0).all() and sides.min() >= 64 and sides.max() <= 8192
    d = np.array([r.density for r in reqs])
    assert d.min() >= 0.1 and d.max() <= 0.6
    g = np.array([r.gens for r in reqs])
    assert g.min() >= 10 and g.max() <= 100000
    # log-uniform generations: the median is near the geometric mean of the range
    assert abs(np.log(np.median(g)) - 0.5 * (np.log(10) + np.log(1e5))) < 0.3
    assert synth.request_stream(n, rate)[123] == reqs[123]      # deterministic
    assert len({r.seed for r in reqs}) == n                     # distinct board seeds


def test_glider_band_lattice():
    band = synth.GliderBand(b0=64, band_rows=512, n=4, spacing=16, off_r=100, off_c=64)
    w = synth.glider_band_words(1024, 4, 5, band)
    cells = oracle.unpack_words(w)
    rc = band.glider_cells(0)
    assert cells[64:64 + 512].sum() == len(rc) == 4 * 4 * 5
    assert all(cells[r, c] for r, c in rc)


def test_oracle_trajectories_fixture():
    # regression fixture written by tests/golden/make_golden.py
    for ln in read_golden("oracle_trajectories.txt"):
        head, pops = ln.split(":")
        R, C, p, seed, torus = head.split()
        b = synth.bernoulli_board(int(R), int(C), float(p), int(seed))
        want = [int(v) for v in pops.split()]
        for g in range(len(want)):
            assert oracle.population(b) == want[g], (head, g)
            b = oracle.step(b, torus=bool(int(torus)))
