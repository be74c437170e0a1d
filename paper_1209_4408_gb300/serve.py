"""Continuous-batching request loop for Game of Life simulations.

Requests (a board, its initial cells, a generation count) arrive over time.
The server keeps every admitted board resident on the device, admits waiting
requests in arrival order while their two device buffers fit the memory
budget, and advances all admitted boards together, one ``gol_step_batch``
launch per tick.  Each tick gives every active board a quantum of
generations (at most what it still needs), sized so that a tick lasts about
``tick_target_s`` of device time (10 ms: on the bench's stream ticks of 10
to 80 ms give the same throughput within 2 %, and the shortest halve the
median latency).  Every board of a tick gets the same quantum, so their
chains of passes are about equally long and the launch stays dense (giving
small boards more generations, up to what their chain covers in a tick,
made the ticks chain-bound: 46 - 69 % of the rate on the bench's stream).
The stepping itself is the library's persistent launch, so the result of
every request is bit-identical to stepping it alone.

The loop never waits for the device while there is something to queue:
ticks are launched ahead (up to ``depth`` in flight on the library's
stream).  The host knows which boards a tick finishes when it launches it
(each board's remaining generations are host state), so a finished board's
result copy is queued right behind that tick and the next tick, without
those boards, is queued right after.  An event recorded behind each tick
tells the host when the tick, and the copies of the boards it finished, are
done; only then are those requests answered, their boards destroyed and
their memory returned to the budget.  Arrivals are admitted between
launches, all those admitted at once as one group (created, their cells
copied into one page-locked buffer that one many-board upload reads in
place), on a side stream, so that the admission runs while the ticks in
flight compute; the next tick launched waits for it and takes the new
boards in.

When the input is closed (every request of the trace has arrived and none
waits for memory), the boards still active get all their remaining
generations in one last launch (``drain``): nothing can join a later tick,
and one launch lets the library's planner split the long runs that are left
into as many units as the device has warps, instead of stepping them tick
by tick behind the largest board.

``serve_fcfs`` is the baseline that serves the same trace one request at a
time with ``gol_step``.
"""
from __future__ import annotations

import collections
import contextlib
import time
from dataclasses import dataclass, field
from typing import Callable, Sequence

import numpy as np

from . import gol


@dataclass
class Job:
    rid: int
    arrival_s: float
    rows: int
    cols: int
    gens: int
    words: np.ndarray                 # initial packed cells (host)
    remaining: int = 0                # generations not yet queued on the device
    handle: int | None = None
    admitted_s: float | None = None
    done_s: float | None = None
    result: np.ndarray | None = None
    staged: object = None             # host memory the upload reads from (kept until retired)
    pending: object = None            # the queued result copy

    @property
    def bytes_on_device(self) -> int:
        return 2 * self.rows * (self.cols // 64) * 8

    @property
    def work(self) -> int:
        return self.rows * self.cols * self.gens


@dataclass
class ServeStats:
    latencies_s: list = field(default_factory=list)
    makespan_s: float = 0.0
    cell_updates: int = 0
    ticks: int = 0
    max_active: int = 0
    max_waiting: int = 0
    peak_bytes: int = 0
    device_s: float = 0.0             # device time of the ticks (0 when the backend cannot tell)

    def summary(self) -> dict:
        lat = np.array(self.latencies_s) if self.latencies_s else np.zeros(1)
        return {
            "requests": len(self.latencies_s),
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3),
            "gcups": self.cell_updates / max(self.makespan_s, 1e-9) / 1e9,
            "makespan_s": self.makespan_s,
            "ticks": self.ticks,
            "max_active": self.max_active,
            "max_waiting": self.max_waiting,
            "peak_device_bytes": self.peak_bytes,
            "device_busy": self.device_s / max(self.makespan_s, 1e-9),
        }


class GpuBackend:
    """The library on the GPU plus the stream plumbing the loop needs:
    ticks, events and result copies on the library's stream (PyTorch's
    current stream, which ``gol.use_torch_allocator`` makes the library's),
    admissions on a side stream, page-locked staging of uploads and
    asynchronous result copies."""

    def __init__(self):
        import torch

        self.torch = torch
        self.stream = torch.cuda.current_stream()
        self.side = torch.cuda.Stream()
        gol.gol_set_stream(self.stream)     # ticks, events and result copies on one stream

    def start(self):
        """Before serving: the side stream waits for the work queued so far."""
        self.side.wait_stream(self.stream)

    @contextlib.contextmanager
    def admission(self):
        """Library calls made inside run on the side stream: the creation
        and upload of new boards overlap the ticks in flight, and the
        library's stream waits for them before its next launch.  The two
        streams share nothing in flight: new boards belong to no queued
        tick, and device memory goes back to the allocator only when idle
        (the library frees boards, plans and staging buffers after an event
        recorded behind their last use; result buffers are kept until their
        tick has completed)."""
        gol.gol_set_stream(self.side)
        try:
            yield
        finally:
            ev = self.torch.cuda.Event()
            ev.record(self.side)
            gol.gol_set_stream(self.stream)
            self.stream.wait_event(ev)

    def gol_create_ex(self, rows, cols, torus, layout):
        return gol.gol_create_ex(rows, cols, torus, layout)

    def gol_set_packed(self, h, words):
        gol.gol_set_packed(h, words)

    def upload_group(self, hs, words_list):
        """Uploads the cells of several new boards with one many-board
        transfer that reads one page-locked buffer in place; returns that
        buffer (to be kept until the upload has run)."""
        n = sum(w.size for w in words_list)
        t = self.torch.empty(n, dtype=self.torch.int64, pin_memory=True)
        flat = t.numpy().view(np.uint64)
        off = 0
        for w in words_list:
            flat[off:off + w.size] = w.reshape(-1)
            off += w.size
        gol.gol_set_packed_batch(hs, flat)
        return t

    def gol_step_batch(self, hs, gens):
        gol.gol_step_batch(hs, gens)

    def gol_destroy(self, h):
        gol.gol_destroy(h)

    def download(self, h, rows, cols):
        """Queues the copy of board h's current state to page-locked host
        memory; the returned object's ``result()`` is valid once an event
        recorded afterwards has completed."""
        torch = self.torch
        n = rows * (cols // 64)
        dev = torch.empty(n, dtype=torch.int64, device="cuda")
        gol.gol_get_packed_device(h, dev.data_ptr(), n)
        host = torch.empty(n, dtype=torch.int64, pin_memory=True)
        host.copy_(dev, non_blocking=True)
        return _Pending(host, rows, cols // 64, dev)

    def record(self):
        ev = self.torch.cuda.Event(enable_timing=True)
        ev.record(self.stream)
        return ev

    def done(self, ev) -> bool:
        return ev.query()

    def wait(self, ev):
        ev.synchronize()

    def elapsed_s(self, a, b) -> float:
        return a.elapsed_time(b) * 1e-3


class _Pending:
    def __init__(self, host, rows, words, dev=None):
        # the device buffer stays allocated until the copy has run (freed
        # earlier, the allocator could hand it to an upload on the side stream)
        self.host, self.shape, self.dev = host, (rows, words), dev

    def result(self) -> np.ndarray:
        return self.host.numpy().view(np.uint64).reshape(self.shape).copy()


@dataclass
class _Tick:
    start: object
    end: object
    finishing: list
    cells_gens: int


class Server:
    def __init__(self, budget_bytes: int = 120 << 30, tick_target_s: float = 0.01,
                 quantum_min: int = 8, quantum_max: int = 1 << 16, keep_results: bool = False,
                 clock: Callable[[], float] = time.perf_counter, backend=None, depth: int = 2,
                 sleep: Callable[[float], None] = time.sleep, poll_s: float = 2e-4, drain: bool = True):
        self.g = backend if backend is not None else GpuBackend()
        self.budget = budget_bytes
        self.tick_target = tick_target_s
        self.qmin, self.qmax = quantum_min, quantum_max
        self.keep = keep_results
        self.clock = clock
        self.depth = max(1, depth)
        self.sleep = sleep
        self.poll = poll_s
        self.drain = drain
        self.quantum = quantum_min
        self.rate_cups = None             # measured cell updates per second of device time
        self._per_gen = 0                 # cells of the boards in the last tick

    def _admit(self, group: list, now: float):
        """Creates the boards of the requests in `group` and queues the upload
        of their cells (one many-board upload when the backend has one, on
        its admission stream when it has one)."""
        ctx = self.g.admission() if hasattr(self.g, "admission") else contextlib.nullcontext()
        with ctx:
            for job in group:
                job.handle = self.g.gol_create_ex(job.rows, job.cols, True, gol.GOL_LAYOUT_PACKED)
                job.remaining = job.gens
                job.admitted_s = now
            if hasattr(self.g, "upload_group"):
                staged = self.g.upload_group([j.handle for j in group], [j.words for j in group])
                for job in group:
                    job.staged = staged
                return
            for job in group:
                self.g.gol_set_packed(job.handle, job.words)

    def _retire(self, job: Job, now: float, stats: ServeStats):
        if job.pending is not None:
            r = job.pending.result()
            job.result = r if self.keep else None
            job.pending = None
        self.g.gol_destroy(job.handle)
        job.handle = None
        job.staged = None
        job.done_s = now
        stats.latencies_s.append(now - job.arrival_s)

    def run(self, jobs: Sequence[Job]) -> ServeStats:
        """Serves ``jobs`` against the clock.  If a library call fails, the
        boards of the admitted requests are released before the error
        propagates."""
        live: list[Job] = []
        try:
            return self._run(jobs, live)
        except BaseException:
            for j in live:
                if j.handle is not None:
                    try:
                        self.g.gol_destroy(j.handle)
                    except Exception:
                        pass
                    j.handle = None
            raise

    def _run(self, jobs: Sequence[Job], live: list) -> ServeStats:
        jobs = sorted(jobs, key=lambda j: j.arrival_s)
        if hasattr(self.g, "start"):
            self.g.start()
        stats = ServeStats()
        waiting: collections.deque = collections.deque()
        inflight: collections.deque = collections.deque()
        active: list[Job] = []            # admitted, generations left to queue
        used = 0
        nxt = 0
        t0 = self.clock()
        while nxt < len(jobs) or waiting or active or inflight:
            # ticks that completed, oldest first: answer the requests they finished
            while inflight and self.g.done(inflight[0].end):
                tk = inflight.popleft()
                now = self.clock() - t0
                for j in tk.finishing:
                    self._retire(j, now, stats)
                    used -= j.bytes_on_device
                    live.remove(j)
                self._observe(tk, stats)
            now = self.clock() - t0
            while nxt < len(jobs) and jobs[nxt].arrival_s <= now:
                waiting.append(jobs[nxt])
                nxt += 1
            group = []
            while waiting and used + waiting[0].bytes_on_device <= self.budget:
                j = waiting.popleft()
                live.append(j)
                group.append(j)
                used += j.bytes_on_device
            if group:
                self._admit(group, now)
                active.extend(group)
            if waiting and not live:
                raise RuntimeError("request %d needs %d bytes, more than the budget" %
                                   (waiting[0].rid, waiting[0].bytes_on_device))
            stats.max_waiting = max(stats.max_waiting, len(waiting))
            stats.max_active = max(stats.max_active, len(active))
            stats.peak_bytes = max(stats.peak_bytes, used)
            if active and len(inflight) < self.depth:
                closed = self.drain and nxt >= len(jobs) and not waiting
                self._launch(active, inflight, stats, closed)
                continue
            if not inflight and not active and nxt < len(jobs):
                # idle until the next arrival
                self.sleep(max(0.0, min(jobs[nxt].arrival_s - (self.clock() - t0), 0.01)))
            elif inflight:
                self.sleep(self.poll)
        stats.makespan_s = self.clock() - t0
        return stats

    def _quanta(self, active: list, closed: bool = False) -> list:
        """Generations of each active board in the next tick: the quantum,
        at most what the board still needs; all it needs once the input is
        closed."""
        if closed:
            return [j.remaining for j in active]
        return [min(j.remaining, self.quantum) for j in active]

    def _launch(self, active: list, inflight: collections.deque, stats: ServeStats, closed: bool = False):
        """One tick: every active board advances by its quantum (at most what
        it still needs); boards that reach their count have their result
        copy queued behind it."""
        q = self._quanta(active, closed)
        cells_gens = sum(j.rows * j.cols * g for j, g in zip(active, q))
        self._per_gen = sum(j.rows * j.cols for j in active)
        start = self.g.record()
        self.g.gol_step_batch([j.handle for j in active], q)
        finishing, still = [], []
        for j, g in zip(active, q):
            j.remaining -= g
            if j.remaining == 0:
                j.pending = self.g.download(j.handle, j.rows, j.cols)
                finishing.append(j)
            else:
                still.append(j)
        active[:] = still
        inflight.append(_Tick(start, self.g.record(), finishing, cells_gens))
        stats.ticks += 1
        stats.cell_updates += cells_gens

    def _observe(self, tk: _Tick, stats: ServeStats):
        """Device time of a completed tick; adapts the quantum so that a tick
        lasts about tick_target_s."""
        dt = self.g.elapsed_s(tk.start, tk.end)
        stats.device_s += dt
        if dt > 0 and tk.cells_gens > 0:
            r = tk.cells_gens / dt
            self.rate_cups = r if self.rate_cups is None else 0.7 * self.rate_cups + 0.3 * r
        self._adapt()

    def _adapt(self):
        if not self.rate_cups or not self._per_gen:
            return
        q = int(self.tick_target * self.rate_cups / max(self._per_gen, 1))
        q = max(self.qmin, min(self.qmax, q))
        self.quantum = max(self.qmin, (q // 8) * 8)


def serve_fcfs(jobs: Sequence[Job], keep_results: bool = False,
               clock: Callable[[], float] = time.perf_counter) -> ServeStats:
    """Baseline: the same trace served one request at a time, in arrival
    order, each with a single gol_step of all its generations."""
    jobs = sorted(jobs, key=lambda j: j.arrival_s)
    stats = ServeStats()
    t0 = clock()
    for j in jobs:
        now = clock() - t0
        if j.arrival_s > now:
            time.sleep(j.arrival_s - now)
        h = gol.gol_create_ex(j.rows, j.cols, True, gol.GOL_LAYOUT_PACKED)
        gol.gol_set_packed(h, j.words)
        gol.gol_step(h, j.gens)
        if keep_results:
            j.result = gol.gol_get_packed(h)
        else:
            gol.gol_sync(h)
        gol.gol_destroy(h)
        j.done_s = clock() - t0
        stats.latencies_s.append(j.done_s - j.arrival_s)
        stats.cell_updates += j.work
        stats.ticks += 1
    stats.makespan_s = clock() - t0
    return stats
