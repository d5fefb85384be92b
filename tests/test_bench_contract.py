"""Host-side parts of bench.py that need no GPU.

* The reference arm (`--impl reference`: the FP64 oracle timed on the host
  cores) prints one JSON line with the fields of the benchmark line: the same
  metric and unit as the GPU arm, a positive rate, an `e2e` object with no
  host-device copies and a `cpu_baseline` describing the oracle sample.
* The recorded DRAM traffic of the dominant kernel is reported only while the
  kernel's sources hash as they did when the counters were taken."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "L6_beta6", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "L6_beta6" and d["config"]["N_sites"] == 72
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]


def test_recorded_traffic_follows_the_source_hash(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    key = ("update", 3, 1152)
    paths, sha, nbytes = bench.CAPTURED_TRAFFIC[key]
    assert nbytes > 0
    monkeypatch.setitem(bench.CAPTURED_TRAFFIC, key, (paths, bench.sources_sha256(paths), nbytes))
    assert bench.captured_traffic(*key) == nbytes
    monkeypatch.setitem(bench.CAPTURED_TRAFFIC, key, (paths, "0" * 64, nbytes))
    assert bench.captured_traffic(*key) is None
    assert bench.captured_traffic("update", 3, 1234) is None
