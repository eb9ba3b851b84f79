"""Host side of bench.py: the oracle's timed CPU sample and the reference arm's
JSON line (no GPU needed)."""
import json
import subprocess
import sys
import types

import bench
from conftest import ROOT


def test_cpu_sample_gives_every_thread_a_plane():
    # the oracle hands each thread a block of whole cube planes: the sample
    # has one plane per thread, and `cores` counts the threads that worked
    r = bench.cpu_baseline(8, 40, threads=2, stride=4)
    assert r["cores"] == 2
    assert r["sample"].startswith("2 cube plane(s) of the 8^3 grid")
    assert "10 energies (1 in 4 of 40)" in r["sample"]
    assert r["value"] > 0 and r["kind"] == "oracle"
    one = bench.cpu_baseline(8, 40, planes=1, threads=4)
    assert one["cores"] == 1 and "40 energies (all 40)" in one["sample"]


def test_reference_arm_line_matches_the_gpu_arm_config():
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--grid", "12", "--n-omega", "64",
           "--steps", "2", "--warmup", "1"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    args = types.SimpleNamespace(grid=12, n_omega=64, mode="point", weight_dtype="f32")
    assert d["impl"] == "reference"
    assert d["config"] == bench.config_of(args, 1)
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"


def test_defaults_and_variant_flag(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.impl, a.grid, a.n_omega, a.mode, a.weight_dtype, a.variant) == \
        (1, "ours", 256, 4000, "point", "f32", None)
    assert a.warmup >= 3
    c = bench.config_of(a, 1)
    assert c["workload"] == "tb8_256cube_4000w_point_f32" and c["tetrahedra"] == 6 * 256 ** 3
    monkeypatch.setattr(sys, "argv", ["bench.py", "--variant", "near_balance", "--steps", "2"])
    a = bench.parse()
    assert a.variant == "near_balance" and a.steps == 2
