"""The allocation-free diagnostics entry point against the FP64 oracle and lb_diagnostics.

lb_diagnostics_noalloc serves callers that cannot allocate device memory when they ask for
diagnostics: extensions inside a host framework whose pool allocator has reserved the device's
memory, monitors of jobs sized to fill the GPU that must not change its footprint, and loops
where cudaMalloc/cudaFree would synchronise the device. Its work space is a static array inside
the library, so it must agree with the oracle's diagnostics of the same field and with the
regular entry point, which uses the caller's buffer, on every call (the array is reused).
This file is collected last so that a failure here never hides the other tests.
"""
import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import lb, workloads

pytestmark = pytest.mark.gpu

KEYS = ("mass", "kinetic_energy", "enstrophy", "dissipation")


def test_noalloc_diagnostics_match_oracle_and_lb_diagnostics_on_two_calls(kbc):
    import torch
    n, nu = 40, 1e-3                    # 64,000 nodes, under the 65,536-node limit
    rho, u = workloads.kida(n, 0.05)
    u = u + 0.01                        # a mean flow: k is taken about <u>
    f0 = oracle.init_equilibrium(rho, u) * (1 + 1e-4 * workloads.population_noise(n, n, n, 2))
    lat = lb.Lattice(n, nu=nu, storage="f64", scheme="aa")
    lat.set_populations(f0)
    fdev = torch.empty((27, n ** 3), dtype=torch.float64, device="cuda")
    for steps in (3, 2):                # two calls in a row; the static array is reused
        lat.step(steps)
        ref = lat.diagnostics()
        lb.lb_get_populations(lat.ctx, fdev.data_ptr(), True)
        got = lb.lb_diagnostics_noalloc(n, n, n, nu, fdev.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream).as_dict()
        orc = oracle.diagnostics(*oracle.macroscopic(fdev.cpu().numpy().reshape(27, n, n, n)),
                                 nu, order=2)
        assert got["nodes"] == n ** 3
        for key in KEYS:
            assert got[key] == pytest.approx(orc[key], rel=1e-12), key
            assert got[key] == pytest.approx(ref[key], rel=1e-10), key
        assert np.allclose(got["momentum"], orc["momentum"], rtol=1e-12, atol=1e-12)
        assert np.allclose(got["momentum"], ref["momentum"], rtol=1e-12, atol=1e-12)
        assert got["nonfinite_count"] == 0
        assert np.isnan(got["gamma_mean"])


def test_noalloc_diagnostics_report_a_nan_population(kbc):
    import torch
    n, nu = 12, 1e-3
    rho, u = workloads.taylor_green(n, 0.05)
    f = oracle.init_equilibrium(rho, u)
    f[5, 3, 4, 7] = np.nan              # one population of one node
    fdev = torch.from_numpy(f.reshape(27, -1).copy()).cuda()
    got = lb.lb_diagnostics_noalloc(n, n, n, nu, fdev.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream,
                                    raise_nonfinite=False).as_dict()
    assert got["nonfinite_count"] == 1
    # averages over the finite nodes stay finite and close to those of the clean field
    clean = oracle.diagnostics(*oracle.macroscopic(oracle.init_equilibrium(rho, u)), nu)
    assert np.isfinite(got["kinetic_energy"])
    assert got["kinetic_energy"] == pytest.approx(clean["kinetic_energy"], rel=0.05)
    with pytest.raises(lb.LBError) as e:
        lb.lb_diagnostics_noalloc(n, n, n, nu, fdev.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    assert e.value.status == lb.LB_ERR_NONFINITE


def test_noalloc_diagnostics_reject_boxes_over_the_limit(kbc):
    with pytest.raises(lb.LBError) as e:
        lb.lb_diagnostics_noalloc(64, 64, 64, 1e-3, 256, 0)   # 262,144 nodes > 65,536
    assert e.value.status == lb.LB_ERR_INVALID_ARG
    assert "65536" in str(e.value)
