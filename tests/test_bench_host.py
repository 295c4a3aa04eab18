"""Host-side pieces of bench.py, without a GPU: the algorithmic bytes of a
step against their closed form (151 B per cell update for the 256^3 patch:
the ghosted state read once and the interior written once, 9 float64
variables, plus the flux registers), and the reference arm's JSON line
(the CPU oracle timed on a bounded sample) with the keys the line must
carry."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_closed_form():
    sys.path.insert(0, ROOT)
    import bench
    n = 256
    per_cell = bench.algorithmic_bytes(n) / n ** 3
    # 72 ((n + 8)^3 + n^3) / n^3 = 150.96, registers 6 * 9 * 8 * 2 / n = 3.4
    assert per_cell == pytest.approx(72 * (264 ** 3 + 256 ** 3) / 256 ** 3 + 6 * 9 * 8 * 2 / 256, rel=1e-15)
    assert abs(per_cell - 6 * 9 * 8 * 2 / 256 - 151) < 0.1


def test_reference_arm_json_line():
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "MHD cell-updates/s per CTU step" and d["unit"] == "cell-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "sample" in d["config"] and d["steps"] == 1 and d["warmup"] == 1
