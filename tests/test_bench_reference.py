"""bench.py's reference arm: the FP64 oracle timed on the host cores (CPU).

The arm prints one JSON line with the GPU arm's metric, unit and workload, and
describes itself (impl, cpu_baseline with the cores it used, an e2e entry with
no transfers). Under a multi-rank launch only rank 0 works and prints. Run here
on a tiny sample of the default workload (a few seeded targets).
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2", "--warmup", "1",
           "--ref-targets", "16"] + list(args)
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


@pytest.fixture(scope="module")
def line():
    lines = _run()
    assert len(lines) == 1
    return lines[0]


def test_reference_line_has_the_contract_keys(line):
    import bench
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC
    assert line["unit"] == "solves/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["config"]["workload"] == "spiral_1024_fft"
    assert line["value"] > 0 and line["ms_per_step"] > 0


def test_reference_line_describes_its_cpu_run(line):
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1
    assert cb["value"] == line["value"] and cb["unit"] == line["unit"]
    assert "16 seeded leaf targets" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_rate_is_targets_over_time(line):
    # solves/s = (targets timed / seconds) / targets of one solve
    tps = line["target_cells_per_s"]
    assert tps == pytest.approx(2 * 16 / (2 * line["ms_per_step"] / 1e3), rel=1e-9)
    assert line["value"] == pytest.approx(tps / (1024 * 1024), rel=1e-9)


def test_reference_other_ranks_do_no_work():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
