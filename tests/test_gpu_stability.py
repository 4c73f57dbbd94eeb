"""Linear stability of the time step of the batched workloads.

The time-step rule (es_dg_cfl_dt) gives the paper's step for its N = 4 rising
bubble at C = 0.5, but on unwarped isotropic meshes C = 0.5 lies on the
stability boundary of LSRK(5,4) for N >= 4: there a relative perturbation of
1e-10 grows to overflow within 300 steps at N = 5..7 (and by 1e5 at N = 4),
while C = 0.45 and below damp it for every order.  The server's default
Courant number (ES_DG_SERVER_DEFAULT_CFL = 0.4) is held here to damping a
seeded perturbation of the rising bubble over 300 steps for every order the
batched workloads draw (3, 4, 7) and the orders between.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2605_16684_gb300 import _build, _lib
    _build.build()
    return _lib


@pytest.mark.parametrize("N", [3, 4, 5, 6, 7])
def test_default_courant_number_is_stable_on_unwarped_meshes(lib, N):
    K = 4
    rng = np.random.default_rng(N)
    a = lib.Solver(K, K, K, N, precision="fp64")
    b = lib.Solver(K, K, K, N, precision="fp64")
    a.init_bubble(amp=0.8)
    q = a.get_state()
    qp = q * (1.0 + 1e-10 * rng.standard_normal(q.shape))
    b.set_state(qp)
    dt = a.cfl_dt(0.4)
    a.step(dt, 300)
    b.step(dt, 300)
    a.sync()
    b.sync()
    growth = np.abs(a.get_state() - b.get_state()).max() / np.abs(qp - q).max()
    assert growth < 1.0, growth
