"""The second example's set-up on the GPU: the eq:E0 field on 400^3 starts at Re_lambda close
to 2000 (8th-order gradients on the grid vs the closed form) and KBC runs it stably."""
import pytest

from paper_1507_02518_gb300 import decay

pytestmark = pytest.mark.gpu


def test_e0_field_starts_at_re_lambda_2000_and_runs(kbc):
    res = decay.run(n=400, t_end=0.0125, every=0.0125)     # 500 steps
    c0, c1 = res["curve"][0], res["curve"][-1]
    print("Re_lambda(0) = %.1f, after %d steps %.1f" % (c0["Re_lambda"], res["steps"],
                                                       c1["Re_lambda"]))
    assert c0["Re_lambda"] == pytest.approx(2000.0, rel=0.03)
    assert c0["k"] == pytest.approx(1.5e-4, rel=2e-3)
    assert all(c["nonfinite"] == 0 for c in res["curve"])
    assert c1["k"] < c0["k"]
