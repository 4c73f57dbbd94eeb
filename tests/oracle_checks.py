"""Oracle references for GPU trajectories (test helper, not a test module).

A GPU result is compared with the CPU oracle advanced from the oracle's own
initial state with the same time step (the step is a scalar the caller passes
to both sides, Section 5 fixes only the CFL number):

* FP64 trajectories: relative L2 error per variable <= 1e-12, or no worse than
  three times the plain double oracle's own distance from the long-double
  oracle (on near-hydrostatic states the double oracle is itself ~1e-12 away).
* mixed-precision trajectories: relative L2 error per variable <= 1e-4 in the
  state (the bar for the state after 100 steps), the three momentum
  components against the norm of the momentum vector (a rising bubble starts
  at rest, so a per-component norm is that of round-off), and the same bar for
  the flow, state minus initial state -- the balanced channel jet included
  (measured flow errors after 1 to 100 steps: <= 5e-5 with the channel state at
  rest as background, <= 2e-7 with the jet as a moving background).
"""
from __future__ import annotations

import numpy as np

import oracle as O

CUBE = dict(lo=(0.0, 0.0, 0.0), hi=(1000.0, 1000.0, 1000.0))
CHANNEL = dict(lo=(0.0, 0.0, 0.0), hi=(40000e3, 6000e3, 30e3), periodic=(1, 0, 0))

_cache: dict = {}


def rel_err(a, b):
    return np.array([np.linalg.norm(a[:, v] - b[:, v]) / max(np.linalg.norm(b[:, v]), 1e-300)
                     for v in range(5)])


def mixed_err(a, b):
    """Per variable, momentum components against the momentum vector's norm."""
    mom = np.sqrt(sum(np.linalg.norm(b[:, v]) ** 2 for v in (1, 2, 3)))
    return np.array([np.linalg.norm(a[:, v] - b[:, v]) /
                     max(mom if v in (1, 2, 3) else np.linalg.norm(b[:, v]), 1e-300)
                     for v in range(5)])


def request_oracle(req, precision="double"):
    """Oracle and initial state of a server request (dict as for Server.submit)."""
    kind = req.get("kind", "bubble")
    K, N = tuple(req["K"]), req["N"]
    if kind == "channel":
        o = O.Oracle(*K, N, precision=precision, f0=1e-4, **CHANNEL)
        return o, o.channel()
    o = O.Oracle(*K, N, warp=req.get("warp", 0.0), precision=precision, **CUBE)
    q0 = o.bubble(300.0, req.get("amp", 0.5), req.get("centre", (500.0, 500.0, 350.0)), 250.0,
                  profile="sharp" if kind == "sharp_bubble" else "smooth")
    return o, q0


def _key(req, dt):
    return (req.get("kind", "bubble"), tuple(req["K"]), req["N"], req.get("warp", 0.0),
            req.get("amp", 0.5), tuple(req.get("centre", (500.0, 500.0, 350.0))),
            req["nsteps"], dt, req.get("precision", "fp64"))


def reference(req, dt):
    """(q0, plain double trajectory, long-double trajectory or None) after req['nsteps']."""
    k = _key(req, dt)
    if k not in _cache:
        o, q0 = request_oracle(req)
        q = o.steps(q0, dt, req["nsteps"])
        ql = None
        if req.get("precision", "fp64") == "fp64":
            ol, _ = request_oracle(req, precision="long")
            ql = ol.steps(q0, dt, req["nsteps"])
        _cache[k] = (q0, q, ql)
    return _cache[k]


def check_fp64(q_gpu, q_plain, q_long, what=""):
    e_gpu, e_plain = rel_err(q_gpu, q_long), rel_err(q_plain, q_long)
    ok = (e_gpu <= 1e-12) | (e_gpu <= 3.0 * e_plain)
    assert np.all(ok), (what, e_gpu, e_plain)
    return e_gpu


def _vector_norms(a):
    """Per-variable L2 norms, the three momentum components given the momentum
    vector's norm."""
    n = np.array([np.linalg.norm(a[:, v]) for v in range(5)])
    n[1:4] = np.sqrt((n[1:4] ** 2).sum())
    return n


def check_mixed(q_gpu, q0, q_ref, what=""):
    e_state = mixed_err(q_gpu, q_ref)
    assert np.all(e_state <= 1e-4), (what, "state", e_state)
    f_gpu, f_ref = q_gpu - q0, q_ref - q0
    err = np.array([np.linalg.norm(f_gpu[:, v] - f_ref[:, v]) for v in range(5)])
    e_flow = err / np.maximum(_vector_norms(f_ref), 1e-300)
    assert np.all(e_flow <= 1e-4), (what, "flow", e_flow)
    return e_state, e_flow


def check_request_result(req, q_flat, dt):
    """Check a served or batched result (flat state) against the oracle."""
    q0, q_plain, q_long = reference(req, dt)
    q = np.asarray(q_flat).reshape(q0.shape)
    # the GPU's initial state is the oracle's to 1e-12 (checked by the initial-state tests)
    if req.get("precision", "fp64") == "fp64":
        return check_fp64(q, q_plain, q_long, what=req)
    return check_mixed(q, q0, q_plain, what=req)
