"""The bench's reference arm on the CPU: it times the FP64 oracle on the host cores and
prints one JSON line with the same metric, unit and config (workload, cells) as the CUDA arm. Under
a multi-rank launch rank 0 alone runs it; the other ranks exit 0 without work."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, rank=0, world=1):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_prints_the_contract_line():
    import bench
    lines = _bench("--steps", "3", "--warmup", "3", "--nx", "256", "--ny", "192")
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    import workloads
    # the CUDA arm prints the same config dict for the same workload
    assert d["config"] == bench.bench_config(workloads.shelf_islands(256, 192), 1)
    assert d["config"]["workload"] == "shelf_islands_256x192" and d["config"]["cells"] == 256 * 192
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert abs(d["ms_per_step"] * d["value"] * 1e6 - 256 * 192) < 1e-6 * 256 * 192


def test_reference_arm_runs_on_rank_zero_only():
    assert _bench("--steps", "3", "--warmup", "3", "--nx", "128", "--ny", "96", "--gpus", "2",
                  rank=1, world=2) == []
    lines = _bench("--steps", "3", "--warmup", "3", "--nx", "128", "--ny", "96", "--gpus", "2",
                   rank=0, world=2)
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2

