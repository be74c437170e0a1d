"""Continuous-batching server: host logic on CPU (fake backend) and, on the
GPU, every result equal alone and in the mix."""
import itertools

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def serve_mod():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1209_4408_gb300 import serve

    return serve


class FakeBackend:
    """Records calls; a board is a dict with its remaining generations."""

    def __init__(self):
        self.ids = itertools.count(1)
        self.boards = {}
        self.live_bytes = 0
        self.peak = 0
        self.batches = []

    def gol_create_ex(self, rows, cols, torus, layout):
        h = next(self.ids)
        self.boards[h] = {"rows": rows, "cols": cols, "gen": 0}
        self.live_bytes += 2 * rows * cols // 8
        self.peak = max(self.peak, self.live_bytes)
        return h

    def gol_set_packed(self, h, words):
        assert words.shape == (self.boards[h]["rows"], self.boards[h]["cols"] // 64)

    def upload_group(self, hs, words_list):
        assert len(hs) == len(words_list) and len(set(hs)) == len(hs)
        self.groups = getattr(self, "groups", 0) + 1
        for h, w in zip(hs, words_list):
            self.gol_set_packed(h, w)
        return object()

    def gol_step_batch(self, hs, gens):
        assert len(set(hs)) == len(hs)
        self.batches.append(list(zip(hs, gens)))
        for h, g in zip(hs, gens):
            assert g > 0
            self.boards[h]["gen"] += g

    def gol_sync(self, h):
        pass

    def gol_get_packed(self, h):
        return self.boards[h]["gen"]

    def gol_destroy(self, h):
        b = self.boards.pop(h)
        self.live_bytes -= 2 * b["rows"] * b["cols"] // 8

    # stream plumbing of the event-driven loop: work completes at once
    def download(self, h, rows, cols):
        gen = self.boards[h]["gen"]
        return type("Pending", (), {"result": lambda self_: gen})()

    def record(self):
        return None

    def done(self, ev):
        return True

    def elapsed_s(self, a, b):
        return 0.0


def make_jobs(serve, n, rate, seed=3, side_hi=512, gen_hi=300):
    reqs = synth.request_stream(n, rate, seed=seed, side_hi=side_hi, gen_lo=5, gen_hi=gen_hi)
    return [serve.Job(r.index, r.arrival_s, r.rows, r.cols, r.gens,
                      synth.bernoulli_words(r.rows, r.cols, r.density, r.seed)) for r in reqs]


def test_host_logic_budget_fifo_and_generations(serve_mod):
    fake = FakeBackend()
    jobs = make_jobs(serve_mod, 40, rate=1e6)                  # all arrive at once
    budget = 3 * max(j.bytes_on_device for j in jobs)
    srv = serve_mod.Server(budget_bytes=budget, tick_target_s=1e-4, keep_results=True, backend=fake)
    st = srv.run(jobs)
    assert st.summary()["requests"] == len(jobs)
    assert fake.peak <= budget                                  # admission respects the budget
    assert all(j.result == j.gens for j in jobs)                # every board got exactly its generations
    assert not fake.boards                                      # everything freed
    admitted = sorted(jobs, key=lambda j: j.admitted_s)
    assert [j.rid for j in admitted] == sorted(j.rid for j in jobs)   # FIFO admission
    assert st.max_waiting > 0 and st.ticks > 1


def test_host_logic_admits_arrivals_in_groups(serve_mod):
    # requests that arrive together are created and uploaded as one group
    fake = FakeBackend()
    jobs = make_jobs(serve_mod, 30, rate=1e6)
    st = serve_mod.Server(budget_bytes=1 << 40, tick_target_s=1e-4, backend=fake).run(jobs)
    assert st.summary()["requests"] == 30 and fake.groups < 30 and not fake.boards


def test_host_logic_drains_in_one_launch_once_input_is_closed(serve_mod):
    # once every request has arrived (and none waits for memory) the active
    # boards get all their remaining generations in one launch; before, the
    # quantum; with drain=False the quantum to the end
    clock = TickClock()
    jobs = make_jobs(serve_mod, 20, rate=2000.0, gen_hi=3000)
    fake = ClockedBackend(clock, jobs)
    srv = serve_mod.Server(budget_bytes=1 << 40, tick_target_s=5e-3, quantum_min=8, keep_results=True,
                           clock=clock, backend=fake, sleep=clock.sleep)
    srv.run(jobs)
    assert all(j.result == j.gens for j in jobs) and not fake.boards
    final = fake.batches[-1]
    assert len(final) > 1                                   # several boards finished together
    # the last launch gave boards more generations than any earlier tick's quantum
    assert max(g for _, g in final) > max(g for b in fake.batches[:-1] for _, g in b)
    clock2 = TickClock()
    jobs2 = make_jobs(serve_mod, 20, rate=2000.0, gen_hi=3000)
    fake2 = ClockedBackend(clock2, jobs2)
    srv2 = serve_mod.Server(budget_bytes=1 << 40, tick_target_s=5e-3, quantum_min=8, keep_results=True,
                            clock=clock2, backend=fake2, sleep=clock2.sleep, drain=False)
    srv2.run(jobs2)
    assert all(j.result == j.gens for j in jobs2)
    assert len(fake2.batches) > len(fake.batches)


def test_host_logic_rejects_oversized_request(serve_mod):
    fake = FakeBackend()
    jobs = make_jobs(serve_mod, 3, rate=1e6)
    srv = serve_mod.Server(budget_bytes=16, backend=fake)
    with pytest.raises(RuntimeError):
        srv.run(jobs)


class FailingBackend(FakeBackend):
    """Fails the n-th batch step (as a library error would)."""

    def __init__(self, fail_at):
        super().__init__()
        self.fail_at = fail_at

    def gol_step_batch(self, hs, gens):
        if len(self.batches) + 1 == self.fail_at:
            raise RuntimeError("step failed")
        super().gol_step_batch(hs, gens)


@pytest.mark.parametrize("fail_at", [1, 3])
def test_host_logic_frees_boards_when_a_step_fails(serve_mod, fail_at):
    fake = FailingBackend(fail_at)
    jobs = make_jobs(serve_mod, 12, rate=1e6, gen_hi=200)
    srv = serve_mod.Server(budget_bytes=1 << 30, tick_target_s=1e-4, backend=fake, drain=False)
    with pytest.raises(RuntimeError, match="step failed"):
        srv.run(jobs)
    assert not fake.boards and fake.live_bytes == 0
    assert all(j.handle is None for j in jobs)


class TickClock:
    """Deterministic clock: each reading advances by `dt`, a sleep by its
    length; a batch step occupies the modelled device for `tick` seconds."""

    def __init__(self, dt=1e-5, tick=5e-3):
        self.t, self.dt, self.tick = 0.0, dt, tick
        self.first = None

    def __call__(self):
        self.t += self.dt
        if self.first is None:
            self.first = self.t
        return self.t

    def sleep(self, s):
        self.t += s


class ClockedBackend(FakeBackend):
    """A modelled device stream: a batch step starts when the work queued
    before it has finished and lasts one tick; an event completes when the
    clock passes the point of the stream where it was recorded.  Records,
    per batch step, its start time and the requests in it."""

    def __init__(self, clock, jobs):
        super().__init__()
        self.clock = clock
        self.rid_of_words = {id(j.words): j.rid for j in jobs}
        self.rid_of = {}
        self.ticks = []
        self.free_at = 0.0              # the modelled stream is idle from then on

    def gol_set_packed(self, h, words):
        super().gol_set_packed(h, words)
        self.rid_of[h] = self.rid_of_words[id(words)]

    def gol_step_batch(self, hs, gens):
        start = max(self.clock.t, self.free_at)
        self.ticks.append((start - self.clock.first, {self.rid_of[h] for h in hs}))
        super().gol_step_batch(hs, gens)
        self.free_at = start + self.clock.tick

    def record(self):
        return max(self.clock.t, self.free_at)

    def done(self, ev):
        return self.clock.t >= ev

    def elapsed_s(self, a, b):
        return b - a


def test_host_logic_admits_arrivals_at_the_next_tick(serve_mod):
    """Continuous batching on a deterministic clock: ticks are queued ahead
    (two in flight), so a request that arrives while boards are stepping
    joins the next tick launched (memory permitting) and waits at most two
    ticks plus host time; the modelled device never idles while requests
    remain; every request gets exactly its generations; ticks hold several
    requests at once."""
    clock = TickClock()
    jobs = make_jobs(serve_mod, 30, rate=400.0, gen_hi=400)       # arrivals over ~75 ms; 5 ms ticks
    fake = ClockedBackend(clock, jobs)
    srv = serve_mod.Server(budget_bytes=1 << 40, tick_target_s=5e-3, quantum_min=8, keep_results=True,
                           clock=clock, backend=fake, sleep=clock.sleep)
    st = srv.run(jobs)
    assert st.summary()["requests"] == len(jobs)
    assert all(j.result == j.gens for j in jobs) and not fake.boards
    host = 200 * clock.dt + srv.poll                                # host readings and one poll per tick
    for j in jobs:
        first = next(t for t, rids in fake.ticks if j.rid in rids)
        assert j.arrival_s <= first + 1e-12
        assert first - j.arrival_s <= 2 * clock.tick + host, (j.rid, j.arrival_s, first)
        assert j.arrival_s <= j.admitted_s <= first + 1e-12 and j.done_s >= first + clock.tick - 1e-12
    assert max(len(rids) for _, rids in fake.ticks) > 1 and st.ticks >= 10
    # back to back: once the first request is in, a tick starts as soon as the
    # previous one ends (until the stream runs dry between arrivals)
    starts = [t for t, _ in fake.ticks]
    gaps = [b - (a + clock.tick) for a, b in zip(starts, starts[1:])]
    assert min(gaps) >= -1e-12
    assert sum(g < 1e-9 for g in gaps) >= len(gaps) // 2


@pytest.mark.gpu
def test_served_results_equal_alone_and_oracle(serve_mod):
    from paper_1209_4408_gb300 import gol

    jobs = make_jobs(serve_mod, 24, rate=2000.0)
    srv = serve_mod.Server(budget_bytes=1 << 24, tick_target_s=0.002, keep_results=True)
    st = srv.run(jobs)
    assert st.summary()["requests"] == len(jobs)
    assert st.ticks > 1 and st.max_active > 1                  # boards really shared launches
    for j in jobs:
        h = gol.gol_create_ex(j.rows, j.cols, True, gol.GOL_LAYOUT_PACKED)
        gol.gol_set_packed(h, j.words)
        gol.gol_step(h, j.gens)
        alone = gol.gol_get_packed(h)
        gol.gol_destroy(h)
        assert np.array_equal(j.result, alone), "request %d differs alone and in the mix" % j.rid
        want = oracle.run(oracle.unpack_words(j.words), j.gens)
        assert np.array_equal(oracle.unpack_words(j.result), want), "request %d vs oracle" % j.rid


@pytest.mark.gpu
def test_fcfs_baseline_matches(serve_mod):
    jobs = make_jobs(serve_mod, 8, rate=5000.0, seed=4)
    st = serve_mod.serve_fcfs(jobs, keep_results=True)
    assert st.summary()["requests"] == 8
    for j in jobs:
        want = oracle.run(oracle.unpack_words(j.words), j.gens)
        assert np.array_equal(oracle.unpack_words(j.result), want)


@pytest.mark.gpu
@pytest.mark.slow
def test_bench_stream_served_equals_alone_and_oracle(serve_mod):
    """The request stream the bench serves (its seed, 2000 requests, sides
    up to 8192, 10 to 1e5 generations), offered faster than the device
    steps it and under a 32 MiB budget, so that requests wait for memory
    and share ticks.  Every result equals the request stepped alone with
    gol_step; every request of at most 1e8 cell updates, and a seeded
    sample of 16 between 1e8 and 1e9, also equals the oracle."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    from paper_1209_4408_gb300 import gol

    reqs = synth.request_stream(2000, 2000.0, seed=synth.SEED_SERVE)
    with ThreadPoolExecutor(max(1, os.cpu_count() or 1)) as ex:
        words = list(ex.map(lambda r: synth.bernoulli_words(r.rows, r.cols, r.density, r.seed), reqs))
    jobs = [serve_mod.Job(r.index, r.arrival_s, r.rows, r.cols, r.gens, w) for r, w in zip(reqs, words)]
    st = serve_mod.Server(budget_bytes=32 << 20, keep_results=True).run(jobs)
    s = st.summary()
    assert s["requests"] == len(jobs) and s["max_waiting"] > 0 and s["max_active"] > 1
    assert s["peak_device_bytes"] <= 32 << 20
    for j in jobs:
        h = gol.gol_create_ex(j.rows, j.cols, True, gol.GOL_LAYOUT_PACKED)
        gol.gol_set_packed(h, j.words)
        gol.gol_step(h, j.gens)
        alone = gol.gol_get_packed(h)
        gol.gol_destroy(h)
        assert np.array_equal(j.result, alone), "request %d differs alone and in the mix" % j.rid
    small = [j for j in jobs if j.work <= 10 ** 8]
    mid = [j for j in jobs if 10 ** 8 < j.work <= 10 ** 9]
    sample = [mid[i] for i in np.random.default_rng(2024).permutation(len(mid))[:16]]
    assert len(small) > 500 and len(sample) == 16

    def oracle_equal(j):
        want = oracle.run(oracle.unpack_words(j.words), j.gens)
        return j.rid, bool(np.array_equal(oracle.unpack_words(j.result), want))

    with ThreadPoolExecutor(max(1, os.cpu_count() or 1)) as ex:
        bad = [rid for rid, ok in ex.map(oracle_equal, small + sample) if not ok]
    assert not bad, "requests differing from the oracle: %s" % bad[:10]
