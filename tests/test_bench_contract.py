"""The reference arm of bench.py (the FP64 oracle on a bounded sample of the
workload, host cores only) prints the benchmark's one JSON line: checked here
on the CPU, key by key."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "unit", "dtype", "data"):
        assert isinstance(d[k], str) and d[k]
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["scaling"] in ("weak", "strong")
    assert d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_multicore_oracle_baseline_runs_independent_processes():
    """The host baseline on several cores: independent single-threaded oracle
    processes on copies of a sample; the rate sums their particle-steps over
    the slowest process's time, and cores counts the processes."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    rate, cores, desc = bench.cpu_rate("c1", 32, 1, 2)
    assert cores == 2 and rate > 0 and desc.startswith("2 processes")
    one, c1, _ = bench.cpu_rate("c1", 32, 1, 1)
    assert c1 == 1 and one > 0


def test_push_traffic_record_matches_the_push_sources():
    """roofline.traffic of the benchmark line comes from the committed ncu
    record of the tiled push, and only while the push's sources are the ones
    it was taken on (their SHA-256): an edit to them without a new capture
    turns the field into null.  Checked here so that such an edit shows."""
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "profiles", "push_tiled_traffic.json")) as f:
        rec = json.load(f)
    n = 299_833_365
    t = bench.push_traffic(rec["workload"], n)
    assert t is not None, "push sources changed since profiles/push_tiled_traffic.json was captured"
    assert t == rec["dram_bytes_per_particle"] * n
    assert 52.0 <= rec["dram_bytes_per_particle"] < 60.0     # algorithmic 52 B, a few re-reads
    assert bench.push_traffic("another workload", n) is None
