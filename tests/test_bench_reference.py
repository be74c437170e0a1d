"""bench.py's reference arm (the oracle timed on the host cores) runs
without a GPU: its JSON line carries the contract's keys, names the same
workload as the GPU arm, and ranks other than 0 print nothing."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def run_reference(workload, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload,
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]


@pytest.mark.parametrize("workload", ["batch", "huge"])
def test_reference_line(workload):
    import bench

    lines = run_reference(workload)
    assert len(lines) == 1
    d = lines[0]
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GCUPS" and d["higher_is_better"]
    assert d["config"]["workload"] == bench.workload_specs(workload, 4096)[1]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    if workload == "huge":
        assert "corner" in cb["sample"]                   # a 131072^2 board is timed on a bounded crop


def test_reference_other_ranks_exit_quietly():
    assert run_reference("batch", {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_gpu_decomposition_plan_without_gpu():
    # beside the host decomposition study, the GPU library's own choice for
    # the Table 2 shapes comes from the host-side planner alone: the tuned
    # generations per pass and tile rows, and a unit plan that covers the
    # board (rows of the segments of all units add up to the board's rows)
    import bench
    from paper_1209_4408_gb300 import gol

    out = bench.gpu_decomposition(((60, 120), (120, 240)), (500,))
    assert [e["board"] for e in out] == ["60x120", "120x240"]
    for e, (R, C) in zip(out, ((60, 120), (120, 240))):
        assert (e["gens_per_pass"], e["tile_rows"]) == gol.gol_tune_get(R, C)
        units = gol.gol_plan_units(R, (C + 63) // 64, e["gens_per_pass"], e["tile_rows"])
        assert e["units"] == len(units)
        assert sum(u["r_end"] - u["r0"] for u in units if u["mode"] == 0) == R
