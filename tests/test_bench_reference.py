"""The reference arm of bench.py (the FP64 oracle on the host cores) on the
small workload: one JSON line with the contract's keys. CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                          "zipf_2000x1000", "--steps", "2", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["steps"] == 2 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert cb["sample"] and set(cb["parts_s"]) >= {"csc", "lloyd_step", "pcg_iter"}
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # counts of the oracle's own solve on a workload it can solve
    cfg = d["config"]
    assert cfg["counts_from"] == "oracle solve" and len(cfg["iters_assumed"]) == len(cfg["lambdas"])
    assert all(it > 0 for it in cfg["iters_assumed"])
