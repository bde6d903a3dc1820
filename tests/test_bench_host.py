"""Host-side checks of the benchmark's arithmetic and of its reference arm's
JSON line (no GPU): the algorithmic bytes and flops per streaming launch,
the traffic figure's tie to the kernel sources, the reference arm's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_figures_of_a_launch():
    """Planted 8192 x 8192, r = 50: V's two bf16 planes (4 B per entry), the
    other factor's plane, the updated factor read and written with its
    plane; 2pnr + 2Mr^2 flops."""
    b, f = bench.algorithmic("bf16x3", 8192, 8192, 50)
    assert b == 8192 * 8192 * 4 + 8192 * 50 * 4 + 8192 * 50 * 12 == 274989056
    assert f == 2 * 8192 * 8192 * 50 + 2 * 8192 * 50 * 50 == 6751846400
    b2, f2 = bench.algorithmic("bf16", 8192, 8192, 50)
    assert b2 == 8192 * 8192 * 2 + 8192 * 50 * 2 + 8192 * 50 * 10 and f2 == f


def test_pass_bounds(monkeypatch):
    """Two-pass bound = copy bandwidth / (2 x one launch's bytes), one-pass
    bound twice that, so the one-pass fraction is half the two-pass one."""
    monkeypatch.setattr(bench, "peaks", lambda: {"hbm_gbs": 6000.0, "_source": "test"})
    b, _ = bench.algorithmic("bf16x3", 8192, 8192, 50)
    d = bench.pass_bounds("bf16x3", 8192, 8192, 50, 9000.0)
    assert d["bytes_per_pass"] == b
    assert abs(d["two_pass"]["bound"] - 6000e9 / (2 * b)) < 0.1
    assert abs(d["one_pass"]["bound"] - 6000e9 / b) < 0.1
    assert abs(d["one_pass"]["frac"] - d["two_pass"]["frac"] / 2) < 1e-4


def test_traffic_only_while_the_kernel_sources_match(monkeypatch):
    key = "k_stream_tc/bf16x3/planted_8192x8192_r50"
    stored = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[key]
    monkeypatch.setattr(bench, "kernel_source_digest", lambda k="": stored["kernel_digest"])
    assert bench.read_traffic(key) == stored["traffic_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_digest", lambda k="": "0" * 16)
    assert bench.read_traffic(key) is None


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--workload", "faces"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "updates/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == "faces_361x2429_r10"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
