"""The benchmark's reference arm on CPU: `bench.py --impl reference` times
the oracle on a small scene and prints the contract's JSON line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "0", "--scale", "0.005", "--width", "160", "--height", "96", "--n-poses", "8"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "frames/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_cpu_baseline_sample_and_extras():
    """The CPU-baseline leg on a small scene: the CHUNK_BLEND sample starts
    at the listed poses and the full-detail and plain-scene extras are
    reported."""
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    from paper_2505_23158_gb300 import synth
    scene, cams = synth.workload_outdoor(seed=0, n_poses=8, scale=0.003, width=96, height_px=64)
    args = argparse.Namespace(cpu_budget_s=0.2, width=96, height=64)
    out = bench.cpu_baseline(args, scene, cams)
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] >= 1
    assert out["full_detail_frames_per_s"] > 0 and out["plain_256_frames_per_s"] > 0
    assert "poses 0, 75" in out["sample"]
