"""Benchmark of the GB300 Game of Life library.

Default workload (one "step"): the uneven batch of 4096 toroidal packed
boards -- rows and cols log-uniform in [32, 2048] rounded to multiples of
64, density U(0.1, 0.6), generations log-uniform in [100, 5000] -- advanced
by one gol_step_batch call (one persistent launch).  The headline value is
batched GCUPS (cell updates per second / 1e9); the same line carries the
plain one-board-at-a-time loop measured on a sample of the batch, the
end-to-end figure through host buffers, the roofline of the dominant
kernel, the oracle's CPU throughput and the SM clocks seen while timing.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload batch|single|huge|bytes|decomposition]

``--impl reference`` times the oracle (the plain serial CPU program of
``oracle/``) on a bounded sample of the same workload (boards above 2048^2
cells on a 2048^2 corner) and prints the same metric for the same
``config.workload``.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

INT_OPS_PER_WORD_GEN = 22          # 2 funnel shifts + 20 LOP3 per 64-cell word per generation


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "single", "huge", "masked", "bytes", "decomposition"])
    ap.add_argument("--boards", type=int, default=4096)
    ap.add_argument("--plain-sample", type=int, default=64, help="boards timed in the plain loop")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-probe", action="store_true", help="skip the integer-throughput probe")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the served runs added to the batch line (0 = skip)")
    ap.add_argument("--serve-load", type=float, default=0.7,
                    help="offered load of the served run as a fraction of the measured batched GCUPS")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="also serve the stream at offered loads 0.3 and 0.5")
    ap.add_argument("--no-fcfs", dest="fcfs", action="store_false",
                    help="skip serving the same trace one request at a time (baseline)")
    ap.add_argument("--no-sub", action="store_true", help="skip the single-board sub-lines (16384^2, 131072^2)")
    ap.add_argument("--no-cpu-configs", action="store_true",
                    help="skip the per-configuration serial / OpenMP oracle baselines")
    return ap.parse_args()


PROFILE = os.path.join(ROOT, "profiles", "persistent_step_kernel.txt")
KERNEL_SRC = os.path.join(ROOT, "paper_1209_4408_gb300", "csrc", "wavefront.cuh")


def recorded_traffic(workload: str):
    """DRAM bytes per launch of the step kernel for `workload` as captured by
    ncu (dram__bytes_read.sum + dram__bytes_write.sum), or None when no
    capture was taken of the kernel source as it is now."""
    import hashlib

    try:
        sha = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
        for ln in open(PROFILE):
            parts = ln.split()
            # "traffic <workload> <bytes> sha256 <hash>"
            if len(parts) == 5 and parts[0] == "traffic" and parts[1] == workload and parts[3] == "sha256":
                if parts[4] == sha:
                    return int(parts[2])
    except OSError:
        return None
    return None


def rank_batch(specs, rank: int):
    """Weak scaling: every rank steps its own copy of the batch; rank r > 0
    draws its boards from seeds derived from the rank."""
    if rank == 0:
        return list(specs)
    return [synth.BoardSpec(s.index, s.rows, s.cols, s.density, s.gens, synth.derive_seed(s.seed, rank))
            for s in specs]


def workload_specs(workload: str, nboards: int, rank: int = 0):
    """The boards of a workload and its description, the same for both arms."""
    if workload == "single":
        return ([synth.BoardSpec(0, 16384, 16384, 0.5, 10000, synth.SEED_SINGLE_16K)],
                "single 16384x16384 toroidal packed board, Bernoulli(0.5), 10000 generations")
    if workload == "huge":
        return ([synth.BoardSpec(0, 131072, 131072, 0.5, 1000, synth.SEED_HUGE_128K)],
                "single 131072x131072 toroidal packed board (2 GiB per buffer), Bernoulli(0.5) with a "
                "cleared 4096-row band holding a 64x64 glider lattice, 1000 generations")
    if workload == "masked":
        return ([synth.BoardSpec(0, 16383, 16383, 0.5, 2000, synth.SEED_MASKED)],
                "single 16383x16383 toroidal packed board (neither side a multiple of 64: 256 words per row, "
                "63 columns in the last), Bernoulli(0.5), 2000 generations")
    if workload == "bytes":
        return ([synth.BoardSpec(0, 256, 256, 0.3, 1000, synth.SEED_BYTES_256)],
                "single 256x256 toroidal byte-per-cell board, Bernoulli(0.3), 1000 generations")
    specs = rank_batch(synth.batch_specs(nboards), rank)
    return (specs, "batch of %d uneven toroidal packed boards (rows, cols log-uniform [32, 2048] "
                   "rounded to x64; density U(0.1,0.6); gens log-uniform [100, 5000])" % len(specs))


def max_over_ranks(ms: float, dist, device=None) -> float:
    """The slowest rank's time (the job finishes when the last rank does)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9], parts[4]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU baselines: the oracle (serial, and its OpenMP row decomposition)
# ---------------------------------------------------------------------------
CPU_SAMPLE_SIDE = 2048   # larger boards are timed on a crop of this side (serial oracle)
CROP_NOTE = "; boards above %d^2 cells timed on their top-left %d x %d corner as a torus" % (
    CPU_SAMPLE_SIDE, CPU_SAMPLE_SIDE, CPU_SAMPLE_SIDE)


def oracle_sample_cells(s):
    """Cells of board spec ``s`` for timing the oracle: the whole board, or
    its top-left CPU_SAMPLE_SIDE^2 corner (stepped as a torus of that size;
    the oracle's time per cell does not depend on the board size) when the
    board is larger.  Returns (cells, cropped)."""
    if s.rows * s.cols > CPU_SAMPLE_SIDE * CPU_SAMPLE_SIDE:
        nr, nc = min(s.rows, CPU_SAMPLE_SIDE), min(s.cols, CPU_SAMPLE_SIDE)
        return synth.bernoulli_region(s.rows, s.cols, s.density, s.seed, 0, 0, nr, nc), True
    return synth.bernoulli_board(s.rows, s.cols, s.density, s.seed), False


def spec_cells(s):
    """The full initial cells of board spec ``s`` (uint8)."""
    if s.density == 0.5 and s.cols % 64 == 0:
        import oracle

        out = np.empty((s.rows, s.cols), dtype=np.uint8)
        step = max(1, (1 << 22) // s.cols)
        for r0 in range(0, s.rows, step):
            r1 = min(s.rows, r0 + step)
            out[r0:r1] = oracle.unpack_words(synth.random_words(r1 - r0, s.cols // 64, s.seed, row0=r0))
        return out
    return synth.bernoulli_board(s.rows, s.cols, s.density, s.seed)


def cpu_oracle_sample(specs, seconds: float, threads: int = 1):
    """Times the oracle on boards taken evenly from ``specs`` for a bounded
    number of generations; a board larger than CPU_SAMPLE_SIDE^2 cells is
    timed on its top-left CPU_SAMPLE_SIDE x CPU_SAMPLE_SIDE corner, stepped
    as a torus of that size (the oracle's time per cell does not depend on
    the board size).  Returns (GCUPS, cores, description)."""
    import oracle

    oracle.build()
    pick = specs[:: max(1, len(specs) // 16)][:16]
    done_cells = 0
    t0 = time.perf_counter()
    used = 0
    cropped = False
    for s in pick:
        cells, crop = oracle_sample_cells(s)
        cropped = cropped or crop
        g = min(s.gens, 8)
        t = time.perf_counter()
        if threads == 1:
            oracle.run(cells, g)
        else:
            oracle.run_rows_omp(cells, g, threads)
        used += time.perf_counter() - t
        done_cells += cells.size * g
        if time.perf_counter() - t0 > seconds:
            break
    desc = "%d boards of the workload (every %dth), min(gens, 8) generations each" % (len(pick), max(1, len(specs) // 16))
    if cropped:
        desc += CROP_NOTE
    return done_cells / used / 1e9, threads, desc


def host_facts():
    """Host cores and CPU model, for the CPU baselines."""
    import platform

    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count() or 1, "cpu_model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def cpu_baselines(cfg_seconds: float = 120.0):
    """The oracle on the host cores, on the seeded inputs of the GPU
    workloads: the serial program (one core) and its OpenMP row
    decomposition (Section 2.1) on every core.  256^2 byte board: all 1000
    generations.  16384^2 board: OpenMP 100 generations of the whole board
    (in chunks of 10, stopping early after ``cfg_seconds``), serial on its
    top-left 2048^2 corner for 10 generations.  4096-board batch: 256 boards
    (every 16th), min(gens, 8) generations each (OpenMP) and min(gens, 2)
    (serial).  Returns {config: {"serial": ..., "openmp_rows": ...}}."""
    import oracle

    oracle.build()
    nproc = os.cpu_count() or 1
    out = {}

    def timed(fn):
        t = time.perf_counter()
        fn()
        return time.perf_counter() - t

    # 256 x 256 byte board, Bernoulli(0.3), all 1000 generations
    s = workload_specs("bytes", 1)[0][0]
    c = synth.bernoulli_board(s.rows, s.cols, s.density, s.seed)
    n = c.size * s.gens
    out["bytes_256"] = {
        "serial": {"value": round(n / timed(lambda: oracle.run(c, s.gens)) / 1e9, 5), "cores": 1,
                   "sample": "the whole board, all %d generations" % s.gens},
        "openmp_rows": {"value": round(n / timed(lambda: oracle.run_rows_omp(c, s.gens, nproc)) / 1e9, 5),
                        "cores": nproc, "sample": "the whole board, all %d generations" % s.gens}}
    # 16384^2 board
    s = workload_specs("single", 1)[0][0]
    c = spec_cells(s)
    done, t_omp = 0, 0.0
    x = c
    while done < 100 and t_omp < cfg_seconds:
        t = time.perf_counter()
        x = oracle.run_rows_omp(x, 10, nproc)
        t_omp += time.perf_counter() - t
        done += 10
    crop = np.ascontiguousarray(c[:CPU_SAMPLE_SIDE, :CPU_SAMPLE_SIDE])
    t_ser = timed(lambda: oracle.run(crop, 10))
    out["single_16384"] = {
        "serial": {"value": round(crop.size * 10 / t_ser / 1e9, 5), "cores": 1,
                   "sample": "top-left %d^2 corner as a torus, 10 generations" % CPU_SAMPLE_SIDE},
        "openmp_rows": {"value": round(c.size * done / t_omp / 1e9, 5), "cores": nproc,
                        "sample": "the whole board, %d generations" % done}}
    del c, x, crop
    # 256 boards of the 4096-board batch
    specs = workload_specs("batch", 4096)[0][::16]
    boards = [synth.bernoulli_board(s.rows, s.cols, s.density, s.seed) for s in specs]
    n8 = sum(b.size * min(s.gens, 8) for b, s in zip(boards, specs))
    n2 = sum(b.size * min(s.gens, 2) for b, s in zip(boards, specs))
    t8 = timed(lambda: [oracle.run_rows_omp(b, min(s.gens, 8), nproc) for b, s in zip(boards, specs)])
    t2 = timed(lambda: [oracle.run(b, min(s.gens, 2)) for b, s in zip(boards, specs)])
    out["batch_4096"] = {
        "serial": {"value": round(n2 / t2 / 1e9, 5), "cores": 1,
                   "sample": "256 boards (every 16th), min(gens, 2) generations each"},
        "openmp_rows": {"value": round(n8 / t8 / 1e9, 5), "cores": nproc,
                        "sample": "256 boards (every 16th), min(gens, 8) generations each"}}
    return out


# ---------------------------------------------------------------------------
# served request stream (continuous batching)
# ---------------------------------------------------------------------------
SERVE_WORKLOAD = ("Poisson arrivals; sides log-uniform [32, 8192] rounded to x64; density U(0.1,0.6); "
                  "gens log-uniform [10, 1e5]; the first %d requests of the seeded stream")


def request_words(reqs):
    """Initial cells of every request (generated on all host cores)."""
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max(1, os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda r: synth.bernoulli_words(r.rows, r.cols, r.density, r.seed), reqs))


def stream_jobs(n_req, rate, words, seed=synth.SEED_SERVE):
    """The first n_req requests of the seeded stream at `rate` per second
    (sizes, densities and generation counts do not depend on the rate)."""
    from paper_1209_4408_gb300 import serve

    reqs = synth.request_stream(n_req, rate, seed=seed)
    return [serve.Job(r.index, r.arrival_s, r.rows, r.cols, r.gens, w) for r, w in zip(reqs, words)]


def served_run(n_req, load, capacity_gcups, budget_bytes, words, fcfs=False, seed=synth.SEED_SERVE):
    """Poisson request stream at `load` x the measured batched capacity,
    served by the continuous-batching loop (and, if `fcfs`, the same trace
    served one request at a time)."""
    from paper_1209_4408_gb300 import serve

    probe = synth.request_stream(n_req, 1.0, seed=seed)
    mean_work = sum(r.work for r in probe) / max(1, len(probe))
    rate = load * capacity_gcups * 1e9 / mean_work
    jobs = stream_jobs(n_req, rate, words, seed)
    st = serve.Server(budget_bytes=budget_bytes).run(jobs)
    out = st.summary()
    out.update({"rate_per_s": round(rate, 3), "offered_load": load, "budget_bytes": budget_bytes,
                "offered_gcups": round(load * capacity_gcups, 1), "workload": SERVE_WORKLOAD % n_req})
    if fcfs:
        fj = stream_jobs(n_req, rate, words, seed)
        fs = serve.serve_fcfs(fj).summary()
        out["fcfs"] = {k: fs[k] for k in ("requests", "p50_ms", "p99_ms", "mean_ms", "gcups", "makespan_s")}
        out["fcfs"]["sample"] = "the same %d-request trace, one request at a time with gol_step" % n_req
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def device_bench(gol, specs, layout, steps, warmup, stream, local, barrier=None):
    """Creates the boards of `specs`, times `steps` gol_step_batch calls of
    all of them (after `warmup`), CUDA events on the library's stream, SM
    clocks sampled meanwhile.  Returns (result dict, boards, pinned host
    words or None)."""
    import torch

    pinned, boards = None, []
    if layout == gol.GOL_LAYOUT_PACKED:
        nwords = sum(s.rows * ((s.cols + 63) // 64) for s in specs)
        pinned = torch.empty(nwords, dtype=torch.int64, pin_memory=True)
        host = pinned.numpy().view(np.uint64)
        views = []
        off = 0
        for s in specs:
            n = s.rows * ((s.cols + 63) // 64)
            views.append((s, host[off:off + n].reshape(s.rows, (s.cols + 63) // 64)))
            off += n

        def fill(item):
            s, v = item
            if s.seed == synth.SEED_HUGE_128K:
                synth.glider_band_words(s.rows, s.cols // 64, s.seed, synth.GliderBand(), out=v)
            elif s.cols % 64:
                v[:] = synth.pack_rows(synth.bernoulli_board(s.rows, s.cols, s.density, s.seed))
            elif s.density == 0.5:
                synth.random_words(s.rows, s.cols // 64, s.seed, out=v)
            else:
                v[:] = synth.bernoulli_words(s.rows, s.cols, s.density, s.seed)

        from concurrent.futures import ThreadPoolExecutor

        with ThreadPoolExecutor(max(1, os.cpu_count() or 1)) as ex:
            list(ex.map(fill, views))
        for s, v in views:
            b = gol.Board(s.rows, s.cols, torus=True, layout=layout)
            b.set_packed(v)
            boards.append(b)
    else:
        for s in specs:
            b = gol.Board(s.rows, s.cols, torus=True, layout=layout)
            b.set(synth.bernoulli_board(s.rows, s.cols, s.density, s.seed))
            boards.append(b)
    handle_array = np.array([b.handle for b in boards], dtype=np.uint64)
    gens_array = np.array([s.gens for s in specs], dtype=np.int64)
    torch.cuda.synchronize()
    for _ in range(warmup):
        gol.gol_step_batch(handle_array, gens_array)
    if barrier:
        barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(local) as clk:
        if barrier:
            barrier()
        torch.cuda.synchronize()
        l0 = gol.gol_kernel_launches()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(steps):
            ev[i][0].record(stream)
            gol.gol_step_batch(handle_array, gens_array)
            ev[i][1].record(stream)
        t_end.record(stream)
        launches = gol.gol_kernel_launches() - l0
        if barrier:
            barrier()
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    res = {"ms_total": t_start.elapsed_time(t_end), "step_ms": step_ms, "clocks": clk.summary(),
           "launches": launches, "handles": handle_array, "gens": gens_array,
           "cells_gens": sum(s.rows * s.cols * s.gens for s in specs),
           "words_gens": sum(s.rows * ((s.cols + 63) // 64) * s.gens for s in specs)}
    return res, boards, pinned


def pipelined_e2e(gol, specs, handles_a, gens_array, host_in, pinned, steps, cells_gens, world, barrier):
    """End to end with two batches in flight: a second set of the same
    boards, each set on its own stream; a step uploads its inputs from
    page-locked memory, steps and queues the download of its results
    (gol_get_packed_batch_async), and a set is reused only once its previous
    step's event has completed.  One batch's transfers and start overlap the
    other's step and its tail."""
    import torch

    boards_b = []
    off = 0
    for s in specs:
        n = s.rows * ((s.cols + 63) // 64)
        b = gol.Board(s.rows, s.cols, torus=True, layout=gol.GOL_LAYOUT_PACKED)
        b.set_packed(host_in[off:off + n].reshape(s.rows, -1))
        boards_b.append(b)
        off += n
    sets = [handles_a, np.array([b.handle for b in boards_b], dtype=np.uint64)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [torch.empty(pinned.numel(), dtype=pinned.dtype, pin_memory=True).numpy().view(np.uint64)
            for _ in range(2)]
    events = [None, None]

    def one(i):
        k = i % 2
        if events[k] is not None:
            events[k].synchronize()
        gol.gol_set_stream(streams[k])
        gol.gol_set_packed_batch(sets[k], host_in)
        gol.gol_step_batch(sets[k], gens_array)
        gol.gol_get_packed_batch_async(sets[k], outs[k])
        ev = torch.cuda.Event()
        ev.record(streams[k])
        events[k] = ev

    prev = torch.cuda.current_stream()
    for i in range(4):                          # warm-up: plans, graphs and transfer plans of both sets
        one(i)
    for e in events:
        e.synchronize()
    barrier()
    n = max(4, steps)
    t0 = time.perf_counter()
    for i in range(n):
        one(i)
    for e in events:
        e.synchronize()
    dt = (time.perf_counter() - t0) / n
    gol.gol_set_stream(prev)
    for b in boards_b:
        b.close()
    return {"value": round(cells_gens * world / dt / 1e9, 2), "unit": "GCUPS", "steps": n,
            "h2d_bytes_per_step": int(host_in.nbytes), "d2h_bytes_per_step": int(outs[0].nbytes),
            "ms_per_step": round(dt * 1e3, 3),
            "method": "two sets of the boards on two streams: a step's upload, launch and download overlap the "
                      "other set's step (gol_get_packed_batch_async)"}


def roofline(gol, words_gens, mean_ms, peak_ops, workload):
    """Integer-pipe roofline of the step kernel on the MEAN step time."""
    achieved = words_gens * INT_OPS_PER_WORD_GEN / (mean_ms * 1e-3) / 1e12
    peak = peak_ops / 1e12
    return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "Tops/s",
            "frac": round(achieved / peak, 4), "traffic": recorded_traffic(workload),
            "peak_source": "integer-pipe probe (LOP3/funnel-shift mix) measured in this run",
            "algorithmic_ops_per_launch": words_gens * INT_OPS_PER_WORD_GEN,
            "time": "mean step (CUDA events on the launching stream)"}


def byte_layout_gcups(gol, s, gens):
    """The same board stored one byte per cell (the path such boards took
    before they could be packed), `gens` generations timed after one."""
    import torch

    b = gol.Board(s.rows, s.cols, torus=True, layout=gol.GOL_LAYOUT_BYTES)
    b.set(synth.bernoulli_board(s.rows, s.cols, s.density, s.seed))
    b.step(1)
    b.sync()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    b.step(gens)
    e.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(e)
    b.close()
    return round(s.rows * s.cols * gens / (ms * 1e-3) / 1e9, 2)


def sub_bench(gol, workload, steps, warmup, stream, local, peak_ops):
    """One of the single-board workloads, timed on its own (a sub-object of
    the batch line)."""
    specs, desc = workload_specs(workload, 1)
    res, boards, _ = device_bench(gol, specs, gol.GOL_LAYOUT_PACKED, steps, warmup, stream, local)
    mean = sum(res["step_ms"]) / len(res["step_ms"])
    k, rows = gol.gol_tune_get(specs[0].rows, specs[0].cols)
    out = {"workload": desc, "value": round(res["cells_gens"] / (mean * 1e-3) / 1e9, 2), "unit": "GCUPS",
           "steps": steps, "warmup": warmup, "ms_per_step": round(mean, 3),
           "step_ms": [round(x, 3) for x in res["step_ms"]], "gens_per_pass": k, "tile_rows": rows,
           "gpu_launches": res["launches"], "clocks": res["clocks"],
           "roofline": roofline(gol, res["words_gens"], mean, peak_ops, workload)}
    for b in boards:
        b.close()
    if workload == "masked":
        out["byte_layout_gcups"] = byte_layout_gcups(gol, specs[0], 20)
        out["note"] = ("roofline counts the 22 operations of a whole word; the masked last word adds 5 per word and "
                       "stage; byte_layout_gcups: the same board one byte per cell, 20 generations")
    return out


def run_gpu(args, rank, world, local):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_1209_4408_gb300 as gol

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = gol.use_torch_allocator(local)
    dinfo = gol.gol_device_info()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- workload -----------------------------------------------------------
    specs, workload = workload_specs(args.workload, args.boards, rank)
    layout = gol.GOL_LAYOUT_BYTES if args.workload == "bytes" else gol.GOL_LAYOUT_PACKED
    res, boards, pinned = device_bench(gol, specs, layout, args.steps, args.warmup, stream, local, barrier)
    handles, handle_array, gens_array = [b.handle for b in boards], res["handles"], res["gens"]
    total_cells_gens, total_words_gens = res["cells_gens"], res["words_gens"]
    step_ms = res["step_ms"]
    ms = max_over_ranks(res["ms_total"] / args.steps, dist, "cuda")
    mean_ms = sum(step_ms) / len(step_ms)
    value = total_cells_gens * world / (ms * 1e-3) / 1e9

    def step():
        gol.gol_step_batch(handle_array, gens_array)

    # ---- plain loop: the same boards stepped one at a time -----------------------
    plain = None
    if args.workload == "batch" and args.plain_sample > 0:
        idx = list(range(0, len(specs), max(1, len(specs) // args.plain_sample)))[:args.plain_sample]
        cg = sum(specs[i].rows * specs[i].cols * specs[i].gens for i in idx)
        for i in idx[:4]:
            gol.gol_step(handles[i], specs[i].gens)        # warm-up: plans for single boards
        torch.cuda.synchronize()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in idx:
            gol.gol_step(handles[i], specs[i].gens)
        b_.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b_)
        plain = {"value": cg / (pms * 1e-3) / 1e9, "unit": "GCUPS", "boards": len(idx),
                 "sample": "every %dth board of the batch, each stepped alone with gol_step" %
                           max(1, len(specs) // args.plain_sample)}

    # ---- end to end through host buffers -------------------------------------------
    e2e = None
    if not args.no_e2e:
        e2e_steps = max(1, min(args.steps, 3))
        out_pinned = torch.empty(pinned.numel(), dtype=pinned.dtype, pin_memory=True) if pinned is not None else None
        host = pinned.numpy().view(np.uint64) if pinned is not None else None
        host_out = out_pinned.numpy().view(np.uint64) if out_pinned is not None else None
        if layout == gol.GOL_LAYOUT_PACKED:
            # warm-up of the transfer path (staging buffers come from the caching allocator)
            gol.gol_set_packed_batch(handle_array, host)
            gol.gol_get_packed_batch(handle_array, host_out)
        barrier()
        t0 = time.perf_counter()
        h2d = d2h = 0
        phase = {"upload_ms": 0.0, "step_ms": 0.0, "download_ms": 0.0}
        for _ in range(e2e_steps):
            if layout == gol.GOL_LAYOUT_PACKED:
                # one upload of all boards, the step, one download of all boards
                ta = time.perf_counter()
                gol.gol_set_packed_batch(handle_array, host)
                torch.cuda.synchronize()
                tb = time.perf_counter()
                h2d += host.nbytes
                step()
                torch.cuda.synchronize()
                tc = time.perf_counter()
                gol.gol_get_packed_batch(handle_array, host_out)
                d2h += host_out.nbytes
                td = time.perf_counter()
                phase["upload_ms"] += (tb - ta) * 1e3
                phase["step_ms"] += (tc - tb) * 1e3
                phase["download_ms"] += (td - tc) * 1e3
            else:
                cells = [synth.bernoulli_board(s.rows, s.cols, s.density, s.seed) for s in specs]
                for b, c in zip(boards, cells):
                    b.set(c)
                    h2d += c.nbytes
                step()
                for b in boards:
                    d2h += b.get().nbytes
        barrier()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        e2e = {"value": total_cells_gens * world / e2e_s / 1e9, "unit": "GCUPS",
               "h2d_bytes_per_step": h2d // e2e_steps, "d2h_bytes_per_step": d2h // e2e_steps,
               "ms_per_phase": {k: round(v / e2e_steps, 3) for k, v in phase.items()},
               "method": "one stream: upload, step, download, each step waits for the last"}
        if layout == gol.GOL_LAYOUT_PACKED and args.workload == "batch":
            # the e2e value: two batches in flight (each step still uploads its
            # inputs and downloads its results); the one-stream figure beside it
            pipe = pipelined_e2e(gol, specs, handle_array, gens_array, host, pinned, args.steps,
                                 total_cells_gens, world, barrier)
            serial = e2e
            e2e = dict(pipe)
            e2e["one_stream"] = serial

    # ---- roofline of the dominant kernel (the persistent step kernel) ---------------
    ops = float("nan") if args.no_probe else gol.gol_probe_int_throughput()[0]
    rl = roofline(gol, total_words_gens, mean_ms, ops, args.workload) \
        if layout == gol.GOL_LAYOUT_PACKED else None
    if rl is not None and not (args.boards == 4096 or args.workload != "batch"):
        rl["traffic"] = None
    # the per-class tune table against the library defaults, on the same boards
    tune = None
    if args.workload == "batch" and not args.no_sub:
        def mean_ms(steps=3):
            for _ in range(2):
                step()
            torch.cuda.synchronize()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                step()
            e.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(e) / steps

        gol.gol_tune_reset()
        default_ms = mean_ms()
        from paper_1209_4408_gb300 import autotune

        autotune.load_shipped()
        tuned_ms = mean_ms()
        tune = {"tuned_ms": round(tuned_ms, 3), "default_ms": round(default_ms, 3),
                "gain": round(default_ms / tuned_ms, 4),
                "table": "tune_gb300.json (per-class entries from autotune.tune_batch) vs no entries"}

    out = {
        "metric": "GCUPS batched (gol_step_batch) vs plain per-board loop on 1 GB300",
        "value": round(value, 2), "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64" if layout == gol.GOL_LAYOUT_PACKED else "u8",
        "data": "synthetic (seeded SplitMix64 Bernoulli boards)",
        "config": {"workload": workload, "boards": len(specs), "cell_updates_per_step": total_cells_gens,
                   "l2": "working set (2 buffers per board) larger than L2" if total_cells_gens and
                   sum(s.rows * s.cols // 4 for s in specs) > dinfo["l2_bytes"] else "fits in L2",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "clocks": res["clocks"],
        "gpu_launches": res["launches"],
        "step_ms": [round(x, 3) for x in step_ms],
    }
    if plain:
        out["plain_loop"] = plain
        out["speedup_vs_plain"] = round(value / world / plain["value"], 2)
    if e2e:
        out["e2e"] = e2e
    if rl:
        out["roofline"] = rl
    if tune:
        out["autotune"] = tune
    for b in boards:
        b.close()
    del pinned
    if args.workload == "batch" and not args.no_sub:
        # the single-board workloads, each timed on its own
        out["single"] = sub_bench(gol, "single", min(args.steps, 5), min(args.warmup, 3), stream, local, ops)
        out["huge"] = sub_bench(gol, "huge", min(args.steps, 3), 1, stream, local, ops)
        out["masked"] = sub_bench(gol, "masked", min(args.steps, 5), min(args.warmup, 2), stream, local, ops)
    if args.workload == "batch" and args.serve_requests > 0:
        n = args.serve_requests
        words = request_words(synth.request_stream(n, 1.0, seed=synth.SEED_SERVE))
        cap = value / world
        out["served"] = served_run(n, args.serve_load, cap, 120 << 30, words, fcfs=args.fcfs)
        out["served_load_1"] = served_run(n, 1.0, cap, 120 << 30, words)
        out["served_budget"] = served_run(n, args.serve_load, cap, 32 << 20, words)
        out["served_budget"]["note"] = ("32 MiB budget: a few of the largest boards at a time, so requests wait "
                                        "for memory (a 2 GB budget never binds at this load)")
        if args.serve_sweep:
            keys = ("offered_load", "budget_bytes", "requests", "p50_ms", "p99_ms", "mean_ms", "gcups",
                    "max_active", "max_waiting", "peak_device_bytes", "device_busy")
            out["served_sweep"] = [{k: r[k] for k in keys if k in r} for r in
                                   (served_run(n, load, cap, 120 << 30, words) for load in (0.3, 0.5))]
        del words
    gol.gol_set_allocator(None, None)
    if rank == 0:
        if not args.no_cpu:
            g, cores, desc = cpu_oracle_sample(specs, args.cpu_seconds, 1)
            out["cpu_baseline"] = {"value": round(g, 5), "unit": "GCUPS", "cores": cores, "kind": "oracle",
                                   "sample": desc, "host": host_facts()}
            if args.workload == "batch" and not args.no_cpu_configs:
                out["cpu_baseline"]["configs"] = cpu_baselines()
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_decomposition(args):
    """The paper's Table 2 experiment on the host cores: the oracle's row,
    column and block decompositions (Sections 2.1-2.2) timed at the table's
    board shapes, iteration counts and thread counts."""
    import oracle

    oracle.build()
    nproc = os.cpu_count() or 1
    threads = sorted({t for t in (1, 2, 4, 8, nproc) if t <= nproc})
    rows = []
    for (R, C) in [(60, 120), (120, 240)]:
        cells = synth.bernoulli_board(R, C, 0.3, 14408)
        for iters in (500, 1000, 2000):
            serial = None
            for t in threads:
                m = max(d for d in range(1, int(t ** 0.5) + 1) if t % d == 0)
                for kind, fn in (("rows", lambda c: oracle.run_rows_omp(c, iters, t)),
                                 ("cols", lambda c: oracle.run_cols_omp(c, iters, t)),
                                 ("blocks", lambda c: oracle.run_blocks_omp(c, iters, m, t // m))):
                    t0 = time.perf_counter()
                    fn(cells)
                    dt = time.perf_counter() - t0
                    if serial is None:
                        serial = dt
                    rows.append({"board": "%dx%d" % (R, C), "iterations": iters, "threads": t,
                                 "decomposition": kind, "seconds": round(dt, 4),
                                 "speedup": round(serial / dt, 2),
                                 "gcups": round(R * C * iters / dt / 1e9, 5)})
    print(json.dumps({"metric": "host decomposition study (paper Table 2 shapes)", "cores": nproc,
                      "data": "synthetic Bernoulli(0.3) boards; the paper's figure-3 pattern is not in the text",
                      "rows": rows, "gpu": gpu_decomposition(((60, 120), (120, 240)), (500, 1000, 2000))}),
          flush=True)


def gpu_decomposition(shapes, iterations):
    """Beside the host study: the GPU library's own decomposition of the same
    boards (the autotuner's generations per pass and tile rows for their size
    class, and the unit plan they give: row blocks x word tiles, segments per
    warp), and, when a GPU is present, the same boards stepped on it in the
    default layout and in the packed one (GCUPS over the table's iteration
    counts, CUDA events)."""
    from paper_1209_4408_gb300 import gol

    out = []
    for (R, C) in shapes:
        W = (C + 63) // 64
        k, tr = gol.gol_tune_get(R, C)
        units = gol.gol_plan_units(R, W, k, tr)
        u0 = units[0]
        entry = {"board": "%dx%d" % (R, C), "gens_per_pass": k, "tile_rows": tr, "units": len(units),
                 "plan": ("%d row block(s) of full rows, %d segment(s) of %d rows per warp" % (len(units), u0["S"], u0["H"])
                          if u0["mode"] == 0 else "%d row block(s) x word tiles" % len(units))}
        try:
            import torch

            if torch.cuda.is_available():
                cells = synth.bernoulli_board(R, C, 0.3, 14408)
                for name, layout in (("default", gol.GOL_LAYOUT_AUTO), ("packed", gol.GOL_LAYOUT_PACKED)):
                    b = gol.Board(R, C, layout=layout)
                    b.set(cells)
                    res = {"layout": "bytes" if b.layout == gol.GOL_LAYOUT_BYTES else "packed"}
                    for it in iterations:
                        b.step(it)                  # warm-up: the plan (or graph) of this count
                        b.sync()
                        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        ev0.record()
                        b.step(it)
                        ev1.record()
                        b.sync()
                        ms = ev0.elapsed_time(ev1)
                        res["gcups_%d" % it] = round(R * C * it / (ms * 1e-3) / 1e9, 3)
                    entry[name] = res
                    b.close()
        except ImportError:
            pass
        out.append(entry)
    return out


def run_reference(args, rank, world):
    """The oracle on the host cores: each step a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle

    oracle.build()
    specs, workload = workload_specs(args.workload if args.workload != "decomposition" else "batch", args.boards)
    pick = specs[:: max(1, len(specs) // 8)][:8]
    sampled = [oracle_sample_cells(s) for s in pick]
    boards = [c for c, _ in sampled]
    gens = 2

    def step():
        n = 0
        for c in boards:
            oracle.run(c, gens)
            n += c.size * gens
        return n

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        n += step()
    dt = time.perf_counter() - t0
    v = n / dt / 1e9
    desc = "%d boards taken evenly from the workload, %d generations each per step" % (len(pick), gens)
    if any(crop for _, crop in sampled):
        desc += CROP_NOTE
    out = {"impl": "reference", "metric": "GCUPS batched (gol_step_batch) vs plain per-board loop on 1 GB300",
           "value": round(v, 6), "unit": "GCUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u8", "data": "synthetic (seeded SplitMix64 Bernoulli boards)",
           "config": {"workload": workload, "boards": len(specs),
                      "parallelism": "oracle (serial, one byte per cell) on one host core, bounded sample"},
           "cpu_baseline": {"value": round(v, 6), "unit": "GCUPS", "cores": 1, "kind": "oracle", "sample": desc},
           "e2e": {"value": round(v, 6), "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "decomposition":
        if rank == 0:
            run_decomposition(args)
    else:
        run_gpu(args, rank, world, local)


if __name__ == "__main__":
    main()
