"""The benchmark's reference arm runs on the CPU and prints the one JSON line its contract
asks for (the GPU arm is exercised by the round-end bench on a GB300)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "3"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["steps"] == 3 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_workload_names_parse():
    sys.path.insert(0, ROOT)
    import bench
    import pytest
    w = bench.parse_workload("batch16_f32_aa")
    assert (w["field"], w["nbox"], w["storage"], w["scheme"]) == ("batch", 16, "f32", "aa")
    w = bench.parse_workload("hit64_f16_pull")
    assert (w["field"], w["n"], w["storage"], w["scheme"]) == ("spectrum", 64, "f16", "pull")
    assert bench.parse_workload("kida100_f64_aa")["field"] == "kida"
    for v in [bench.MAIN] + bench.VARIANTS:
        assert bench.parse_workload(v["name"]) == v
    with pytest.raises(SystemExit):
        bench.parse_workload("hit64_bf16_pull")
    a = bench.parse_args(["--variants", "batch16_f32_pull,hit64_f32_aa"])
    assert a.variants == "batch16_f32_pull,hit64_f32_aa" and a.warmup >= 3
