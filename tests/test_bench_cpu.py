"""bench.py's reference arm (the CPU oracle) runs without a GPU and prints one JSON line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "256",
                        "--steps", "2", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "Gcell-updates/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_warmup_is_at_least_three():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "64",
                        "--steps", "1", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    assert json.loads(r.stdout.strip().splitlines()[-1])["warmup"] == 3


def test_batch_roofline_per_class_bound():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    bt = W.batching(ngrids=64)
    r = bench.batch_roofline(bt, 4, 10.0, sms=152, hbm=6000.0)
    cls = r["classes"]
    assert cls["on_chip"]["grids"] + cls["streamed"]["grids"] == 64
    assert abs(cls["on_chip"]["updates"] + cls["streamed"]["updates"] - bt.updates) < 1
    want = (max(cls["on_chip"]["t_hbm_ms"], cls["on_chip"]["t_fp32_lanes_ms"])
            + max(cls["streamed"]["t_hbm_ms"], cls["streamed"]["t_fp32_lanes_ms"]))
    assert abs(r["time_bound_ms"] - want) < 1e-9 and abs(r["frac"] - want / 10.0) < 1e-12
    # the lane time uses the same operations per update as the single-grid roofline
    lanes = cls["streamed"]["updates"] * bench.ALG_OPS_PER_UPDATE / (152 * 128 * 2070e6) * 1e3
    assert abs(cls["streamed"]["t_fp32_lanes_ms"] - lanes) < 1e-9
    # a deeper plan streams fewer bytes for the same updates
    assert bench.batch_roofline(bt, 8, 10.0, sms=152, hbm=6000.0)["classes"]["streamed"]["hbm_bytes"] < \
        cls["streamed"]["hbm_bytes"]


def test_stream_roofline_picks_the_binding_bound():
    sys.path.insert(0, ROOT)
    import bench
    cells = 8192 * 8192
    # depth 8: 14 x 8 operations per cell against 152 x 128 lanes at 2070 MHz
    # take longer than 16 B per cell at 6671 GB/s: the lanes bind
    r = bench.stream_roofline(cells, 8, 0.384, 6671.2, 152, 2070.0)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["alu"]["time_bound_us"] - 14 * 8 * cells / (152 * 128 * 2070e6) * 1e6) < 1e-6
    assert abs(r["frac"] - r["alu"]["time_bound_us"] / 384.0) < 1e-9
    assert abs(r["hbm"]["frac"] - 16 * cells / 0.384e-3 / 6671.2e9) < 1e-9
    # depth 1: HBM binds
    r1 = bench.stream_roofline(cells, 1, 0.168, 6671.2, 152, 2070.0)
    assert r1["bound"] == "hbm" and r1["unit"] == "GB/s" and r1["frac"] == r1["hbm"]["frac"]
