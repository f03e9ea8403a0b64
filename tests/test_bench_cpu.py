"""bench.py's reference arm runs on the host (the CPU oracle) and prints one
JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GB/s"
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    from oracle import cores
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == cores.host_cores()
    assert d["cpu_baseline"]["value"] == d["value"]
    one = d["cpu_baseline"]["one_core"]
    assert one["cores"] == 1 and one["value"] > 0
    assert "workload" in d["config"] and "4096x4096" in d["config"]["workload"]



def test_sweep_team_grid_follows_the_sm_count():
    from paper_2106_03219_gb300 import autotune
    g = autotune.team_grid(152)
    assert list(g) == sorted(set(g))
    for m in (1, 2, 4, 8, 16, 32):
        assert 152 * m in g
    for p in (1024, 2048, 4096, 8192, 16384):
        assert p in g
    assert 148 not in g and 1184 not in g
