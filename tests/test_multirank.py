"""The N > 1 path of bench.py (one process per GPU, weak scaling, no
data-path collective) exercised as two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = bench.rank_batch(synth.batch_specs(32), rank)
    seeds = torch.tensor([s.seed % (1 << 62) for s in specs], dtype=torch.int64)
    gathered = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    ms = bench.max_over_ranks(10.0 + rank, dist)
    if rank == 0:
        out.put((ms, [g.tolist() for g in gathered], [(s.rows, s.cols, s.gens) for s in specs]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_host_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    ms, seeds, shapes = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert ms == 11.0                                    # the slower rank's time
    assert not set(seeds[0]) & set(seeds[1])             # ranks step different boards
    import synth

    assert shapes == [(s.rows, s.cols, s.gens) for s in synth.batch_specs(32)]   # same shapes: weak scaling
