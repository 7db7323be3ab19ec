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


def test_roofline_arithmetic_and_the_kernel_hash(tmp_path, monkeypatch):
    """achieved = algorithmic bytes per update x updates per second; frac = achieved / peak;
    the hash that keys the ncu traffic figure moves with the kernel sources, the kernel
    selection and the launch code alike."""
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    r = bench.roofline("f32", 30000.0, 6789.6, "measured", traffic=3.58e9)
    assert r["achieved"] == round(216 * 30000e6 / 1e9, 1)
    assert abs(r["frac"] - r["achieved"] / 6789.6) < 1e-4
    assert r["traffic"] == 3.58e9 and r["peak_source"] == "of measured" and r["bound"] == "hbm"
    assert bench.roofline("f16", 1000.0, 1000.0, "fallback")["achieved"] == 108.0
    assert {"kbc_device.cuh", "kbc_kernels.cuh", "kbc_ops.h", "lb_api.cu"} <= set(
        bench.KERNEL_SOURCES)
    src = os.path.join(ROOT, "paper_1507_02518_gb300", "csrc")
    dst = tmp_path / "paper_1507_02518_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    assert h0 == bench.kernel_source_hash()
    for name in ("lb_api.cu", "kbc_ops.h", "kbc_device.cuh"):
        with open(dst / name, "a") as fh:
            fh.write("\n")
        h1 = bench.kernel_source_hash()
        assert h1 != h0, name
        h0 = h1
