"""Streaming alone is an exact permutation. With LBGK (gamma = 2) and nu = 1e30 the relaxation
rate beta = 1/(6 nu + 1) is ~1e-31, so each collision changes no stored value and a step is the
propagation of eq:Egeneral only: f_i(x, t + n) = f_i(x - n v_i, t), bit for bit, in every
storage, scheme and kernel."""
import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import lb, workloads

from test_gpu_parity import lattice

pytestmark = pytest.mark.gpu

V, W = oracle.lattice()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("kind", ["direct", "packed", "staged", "persistent", "rows", "adj"])
# the packed kernel takes blocks of whole rows for nx = 128, 256, 512 (2, 4 and 2 x 4 warps)
# and blocks of consecutive nodes straddling rows for the others; the rows kernel takes tiles
# of 4, 2 and 1 whole rows for nx = 64, 128 (ny = 4), 256 and 256-node segments for 512
@pytest.mark.parametrize("shape", [(10, 9, 8), (37, 5, 4), (3, 3, 3), (300, 3, 4), (128, 3, 5),
                                   (256, 4, 3), (512, 3, 3), (64, 4, 3), (128, 4, 3)])
@pytest.mark.parametrize("steps", [1, 4, 7])
def test_streaming_is_an_exact_permutation(kbc, storage, scheme, kind, shape, steps):
    nx, ny, nz = shape
    lat = lattice(shape, nu=1e30, storage=storage, scheme=scheme, gamma="lbgk")
    try:
        lat.set_kernel(kind)
    except lb.LBError as e:
        assert e.status == lb.LB_ERR_UNSUPPORTED
        pytest.skip("kernel %s not built for %s with nx = %d" % (kind, storage, nx))
    f0 = W.reshape(27, 1, 1, 1) * (1.0 + 0.01 * workloads.population_noise(nx, ny, nz, 5))
    lat.set_populations(f0)
    start = lat.get_populations()              # the stored (rounded) state
    lat.step(steps)
    got = lat.get_populations()
    expect = np.empty_like(start)
    for i in range(27):
        vx, vy, vz = V[i]
        expect[i] = np.roll(start[i], shift=(steps * vz, steps * vy, steps * vx), axis=(0, 1, 2))
    assert np.array_equal(got, expect)
