"""Error of FP32 and FP16 storage against FP64 storage on the same workload (GPU, C ABI).

64^3 random-spectrum field (k0 = 4, u_rms = 0.04, nu = 2e-4), 200 steps, diagnostics every 20.
Measured on GB300: FP32 k 2.8e-6, eps 3.8e-6 (relative), velocity rms 3.6e-6 (relative);
FP16 k 1.8e-5, eps 2.6e-5, velocity rms 1.3e-3. The bounds leave a factor of about 5.
"""
import pytest

from paper_1507_02518_gb300 import precision

pytestmark = pytest.mark.gpu


def test_reduced_precision_error_against_fp64(kbc):
    res = precision.study(n=64, steps=200, every=20, field="spectrum", nu=2e-4,
                          precisions=(("f32", "pull"), ("f16", "aa")))
    f32 = res["results"]["f32_pull"]
    f16 = res["results"]["f16_aa"]
    assert f32["nonfinite"] == 0 and f16["nonfinite"] == 0
    assert f32["kinetic_energy_max_rel_err"] < 2e-5
    assert f32["dissipation_max_rel_err"] < 2e-5
    assert f32["velocity_rms_rel_err"] < 2e-5
    assert f16["kinetic_energy_max_rel_err"] < 1e-4
    assert f16["dissipation_max_rel_err"] < 1.5e-4
    assert f16["velocity_rms_rel_err"] < 7e-3
