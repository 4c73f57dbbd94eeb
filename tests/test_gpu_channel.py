"""The channel (periodic x, walls y and z, f-plane Coriolis, balanced zonal jet plus a
Gaussian wind perturbation) advanced on the GPU against the oracle.

* FP64, 25 steps: the state per variable within 1e-12 of the long-double oracle's
  trajectory, or no worse than three times the plain double oracle's own distance from
  it (the rule of the other FP64 trajectory tests; the long-double oracle is software
  quad precision on some hosts, hence the shorter run).
* mixed, 100 steps: the state and the flow (state minus initial state) within 1e-4 per
  variable (momentum against the momentum vector's norm: the jet makes rho v and rho w
  tiny next to rho u), with the channel state at rest as background (the server's
  batched kernels; measured flow errors <= 7e-6) and with the balanced jet itself as a
  moving background (<= 3e-7).
* mass is conserved to round-off (periodic x, reflecting walls).
"""
import numpy as np
import pytest

import oracle as O
from oracle_checks import check_fp64, check_mixed

pytestmark = pytest.mark.gpu

M = dict(lo=(0.0, 0.0, 0.0), hi=(40000e3, 6000e3, 30e3), periodic=(1, 0, 0))
K = (6, 3, 2)
NSTEPS = {"fp64": 25, "mixed": 100, "jet": 100}


@pytest.fixture(scope="module")
def lib():
    from paper_2605_16684_gb300 import _build, _lib
    _build.build()
    return _lib


_refs = {}


def oracle_trajectory(n):
    if n not in _refs:
        o = O.Oracle(*K, 4, f0=1e-4, **M)
        q0 = o.channel()
        dt = o.cfl_dt(q0, 0.5)
        _refs[n] = (q0, dt, o.steps(q0, dt, n))
    return _refs[n]


@pytest.mark.parametrize("case,mass_bar", [("fp64", 1e-13), ("mixed", 1e-10), ("jet", 1e-10)])
def test_channel_steps(lib, case, mass_bar):
    n = NSTEPS[case]
    q0, dt, ref = oracle_trajectory(n)
    precision = "fp64" if case == "fp64" else "mixed"
    s = lib.Solver(*K, 4, precision=precision, f0=1e-4, **M)
    s.init_channel(background="jet" if case == "jet" else "rest")
    assert np.abs(s.get_state() - q0).max() <= 1e-12 * np.abs(q0).max()
    m0 = s.integrals()[0]
    s.step(dt, n)
    s.sync()
    q = s.get_state()
    if precision == "fp64":
        ref_long = O.Oracle(*K, 4, f0=1e-4, precision="long", **M).steps(q0, dt, n)
        check_fp64(q, ref, ref_long, what="channel")
    else:
        e_state, e_flow = check_mixed(q, q0, ref, what=case)
        print(case, "state", e_state, "flow", e_flow)
    assert abs(s.integrals()[0] - m0) <= mass_bar * abs(m0)
