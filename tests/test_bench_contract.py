"""The reference arm of bench.py (the float64 oracle timed on the host cores) keeps the
benchmark line's contract without a GPU: one JSON line with our arm's metric, unit,
direction and workload config, a bounded-sample `cpu_baseline` and an `e2e` object without
host-device copies; under torchrun only rank 0 runs and prints.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from workloads import config  # noqa: E402


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "1", "--ref-seconds", "1", *args]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_line_keeps_the_contract():
    out = _run()
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    wl = config("L256")
    assert d["impl"] == "reference"
    assert d["metric"] == bench.metric_name(wl)
    assert d["unit"] == "accepted/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1
    assert d["config"] == bench.workload_config(wl, 1)     # our arm's workload keys
    assert d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "rows timed" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


@pytest.mark.parametrize("rank", ["1", "3"])
def test_reference_other_ranks_exit_without_work(rank):
    out = _run({"RANK": rank, "WORLD_SIZE": "4", "LOCAL_RANK": rank})
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""
