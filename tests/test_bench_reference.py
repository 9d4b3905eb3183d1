"""bench.py's reference arm (the CPU oracle on the bench workload) keeps its JSON-line contract (no GPU).

Run on the small ER workload: one line with impl "reference", the main line's metric and workload
config, a positive steps/s value, a cpu_baseline describing the run and an e2e block without host
copies; under a multi-rank launch only rank 0 prints.
"""
import json
import os
import subprocess
import sys

from tests.conftest import ROOT


def _run(extra_env=None):
    env = dict(os.environ, **(extra_env or {}))
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, env=env, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_reference_line():
    import bench

    lines = _run()
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC_MAIN
    assert line["unit"] == "steps/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    cfg = line["config"]
    assert cfg["walkers"] == 1024 and cfg["length"] == 80 and cfg["updates_per_step"] == 2048
    assert "1024 of the 1024 walkers" in cfg["sample"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_other_ranks_print_nothing():
    assert _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}) == []
