"""The reference arm of bench.py on the host: the CPU oracle's whole job
(build of all rows, search of all queries) per timed step, printed as one
JSON line with the fields the benchmark contract names (impl, metric, unit,
the e2e object with no copies, the cpu_baseline that describes the run)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n-db", "20000",
         "--nq", "200", "--steps", "2", "--warmup", "3"],
        cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "queries/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and abs(d["value"] - 200 / (d["ms_per_step"] / 1000.0)) < 1e-6 * d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "20000 rows" in cb["sample"] and "200 queries" in cb["sample"]
    assert d["config"]["n_db"] == 20000 and d["config"]["nq"] == 200
