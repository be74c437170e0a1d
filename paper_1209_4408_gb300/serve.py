"""Continuous-batching request loop for Game of Life simulations.

Requests (a board, its initial cells, a generation count) arrive over time.
The server keeps every admitted board resident on the device, admits waiting
requests in arrival order while their two device buffers fit the memory
budget, and advances all admitted boards together, one
``gol_step_batch`` launch per tick.  Each tick gives every active board a
quantum of generations (at most what it still needs); the quantum adapts so
that a tick lasts about ``tick_target_s``.  Requests that arrive while a tick
runs are admitted (created and uploaded) before the next tick; boards that
reach their generation count are read back and freed at the end of the tick
that finished them.  The stepping itself is the library's persistent launch,
so the result of every request is bit-identical to stepping it alone.

``serve_fcfs`` is the baseline that serves the same trace one request at a
time with ``gol_step``.
"""
from __future__ import annotations

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
    remaining: int = 0
    handle: int | None = None
    admitted_s: float | None = None
    done_s: float | None = None
    result: np.ndarray | None = None

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
        }


class Server:
    def __init__(self, budget_bytes: int = 120 << 30, tick_target_s: float = 0.02,
                 quantum_min: int = 8, quantum_max: int = 1 << 16, keep_results: bool = False,
                 clock: Callable[[], float] = time.perf_counter, backend=None):
        self.g = backend if backend is not None else gol
        self.budget = budget_bytes
        self.tick_target = tick_target_s
        self.qmin, self.qmax = quantum_min, quantum_max
        self.keep = keep_results
        self.clock = clock
        self.quantum = quantum_min
        self.rate_cups = None             # measured cell updates per second

    def _admit(self, job: Job, now: float):
        job.handle = self.g.gol_create_ex(job.rows, job.cols, True, gol.GOL_LAYOUT_PACKED)
        self.g.gol_set_packed(job.handle, job.words)
        job.remaining = job.gens
        job.admitted_s = now

    def _retire(self, job: Job, now: float, stats: ServeStats):
        if self.keep:
            job.result = self.g.gol_get_packed(job.handle)
        else:
            self.g.gol_sync(job.handle)
        self.g.gol_destroy(job.handle)
        job.handle = None
        job.done_s = now
        stats.latencies_s.append(now - job.arrival_s)

    def run(self, jobs: Sequence[Job]) -> ServeStats:
        """Serves ``jobs`` (sorted by arrival) against the wall clock.  If a
        library call fails, the boards of the admitted requests are freed
        before the error propagates."""
        active: list[Job] = []
        try:
            return self._run(jobs, active)
        except BaseException:
            for j in active:
                if j.handle is not None:
                    try:
                        self.g.gol_destroy(j.handle)
                    except Exception:
                        pass
                    j.handle = None
            raise

    def _run(self, jobs: Sequence[Job], active: list) -> ServeStats:
        jobs = sorted(jobs, key=lambda j: j.arrival_s)
        stats = ServeStats()
        waiting: list[Job] = []
        used = 0
        nxt = 0
        t0 = self.clock()
        while nxt < len(jobs) or waiting or active:
            now = self.clock() - t0
            while nxt < len(jobs) and jobs[nxt].arrival_s <= now:
                waiting.append(jobs[nxt])
                nxt += 1
            while waiting and used + waiting[0].bytes_on_device <= self.budget:
                j = waiting.pop(0)
                active.append(j)
                self._admit(j, now)
                used += j.bytes_on_device
            if waiting and not active:
                raise RuntimeError("request %d needs %d bytes, more than the budget" %
                                   (waiting[0].rid, waiting[0].bytes_on_device))
            stats.max_waiting = max(stats.max_waiting, len(waiting))
            stats.max_active = max(stats.max_active, len(active))
            stats.peak_bytes = max(stats.peak_bytes, used)
            if not active:
                if nxt < len(jobs):                       # idle until the next arrival
                    time.sleep(max(0.0, min(jobs[nxt].arrival_s - (self.clock() - t0), 0.01)))
                continue
            # one tick: every active board advances by min(remaining, quantum)
            q = [min(j.remaining, self.quantum) for j in active]
            cells_gens = sum(j.rows * j.cols * g for j, g in zip(active, q))
            t_tick = self.clock()
            self.g.gol_step_batch([j.handle for j in active], q)
            # admit arrivals while the tick runs (uploads queue behind it)
            now = self.clock() - t0
            while nxt < len(jobs) and jobs[nxt].arrival_s <= now:
                waiting.append(jobs[nxt])
                nxt += 1
            self.g.gol_sync(active[0].handle)
            dt = self.clock() - t_tick
            stats.ticks += 1
            stats.cell_updates += cells_gens
            now = self.clock() - t0
            still = []
            for j, g in zip(active, q):
                j.remaining -= g
                if j.remaining == 0:
                    self._retire(j, now, stats)
                    used -= j.bytes_on_device
                else:
                    still.append(j)
            active[:] = still
            self._adapt(cells_gens, dt, active)
        stats.makespan_s = self.clock() - t0
        return stats

    def _adapt(self, cells_gens: int, dt: float, active: Sequence[Job]):
        if dt > 0 and cells_gens > 0:
            r = cells_gens / dt
            self.rate_cups = r if self.rate_cups is None else 0.7 * self.rate_cups + 0.3 * r
        if not active or not self.rate_cups:
            return
        per_gen = sum(j.rows * j.cols for j in active)
        q = int(self.tick_target * self.rate_cups / max(per_gen, 1))
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
