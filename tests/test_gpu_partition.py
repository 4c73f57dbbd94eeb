"""Domain decomposition on one GPU: a mesh cut into slabs of x element layers,
each slab its own handle, traces exchanged before every stage.

The slabs' geometry, right-hand sides and LSRK steps equal the whole mesh's bit
for bit (the same node positions, face geometry and per-face arithmetic; only
the source of the outside state at a cut changes), in FP64 and in mixed
precision, with periodic and walled x, ragged and single-layer slabs, a warped
mesh, and the channel with its Coriolis term.  Each slab result is also held
to the CPU oracle directly: right-hand sides to 1e-12 per variable, FP64
trajectories to 1e-12 or the long-double floor, mixed trajectories to 1e-4 per
variable (see oracle_checks).
"""
import numpy as np
import pytest

import oracle as O
from oracle_checks import check_fp64, check_mixed, rel_err
from paper_2605_16684_gb300 import inputs
from paper_2605_16684_gb300._lib import EsDgError

pytestmark = pytest.mark.gpu

CUBE = dict(lo=(0.0, 0.0, 0.0), hi=(1000.0, 1000.0, 1000.0))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_16684_gb300 import _build, _lib
    _build.build()
    return _lib


CASES = [
    # K, N, bounds or P, periodic, warp
    ((4, 3, 2), 3, 2, (1, 1, 0), 0.0),
    ((5, 2, 3), 4, [(0, 1), (1, 3), (3, 5)], (1, 1, 0), 0.05),
    ((5, 2, 3), 4, [(0, 2), (2, 5)], (0, 1, 0), 0.05),
    ((3, 2, 2), 2, 3, (1, 0, 0), 0.0),
    ((4, 2, 2), 7, 2, (1, 1, 0), 0.05),
]


def pair(lib, K, N, parts, periodic, warp, precision="fp64", **kw):
    mesh = dict(CUBE, periodic=periodic, warp=warp)
    mesh.update(kw.pop("mesh", {}))
    whole = lib.Solver(*K, N, precision=precision, **mesh, **kw)
    split = lib.PartitionedSolver(*K, N, P=parts if isinstance(parts, int) else 2,
                                  bounds=None if isinstance(parts, int) else parts,
                                  precision=precision, **mesh, **kw)
    return whole, split, mesh


@pytest.mark.parametrize("K,N,parts,periodic,warp", CASES)
def test_slab_geometry_equals_whole(lib, K, N, parts, periodic, warp):
    whole, split, _ = pair(lib, K, N, parts, periodic, warp)
    xw, Jw, Jaw = whole.geometry()
    g = lambda a: a.reshape(K[2], K[1], K[0], *a.shape[1:])
    for s, (b, e) in zip(split.parts, split.bounds):
        xs, Js, Jas = s.geometry()
        for w, p in ((xw, xs), (Jw, Js), (Jaw, Jas)):
            assert np.array_equal(g(w)[:, :, b:e].reshape(p.shape), p)


@pytest.mark.parametrize("K,N,parts,periodic,warp", CASES)
def test_slab_rhs_equals_whole(lib, K, N, parts, periodic, warp):
    whole, split, mesh = pair(lib, K, N, parts, periodic, warp)
    o = O.Oracle(*K, N, **mesh)
    x, _, _ = o.geometry()
    q = inputs.perturb_state(o.bubble(), x, mesh["lo"], mesh["hi"], seed=7)
    r = split.rhs(q)
    assert np.array_equal(r, whole.rhs(q))
    err = rel_err(r, o.rhs(q))
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("K,N,parts,periodic,warp", CASES[:3])
def test_slab_steps_equal_whole(lib, K, N, parts, periodic, warp, precision):
    whole, split, _ = pair(lib, K, N, parts, periodic, warp, precision=precision)
    whole.init_bubble(amp=0.8, profile="sharp")
    split.init_bubble(amp=0.8, profile="sharp")
    q_init = split.get_state()
    assert np.array_equal(q_init, whole.get_state())
    dt = whole.cfl_dt(0.5)
    assert split.cfl_dt(0.5) == dt
    whole.step(dt, 4)
    # one call of one step (issued directly), then a call of three (the first issued,
    # two replays of the captured step): consecutive calls reuse the ordering events
    split.step(dt, 1)
    split.step(dt, 3)
    q = split.get_state()
    assert np.array_equal(q, whole.get_state())
    oracle_trajectory(q, q_init, precision, dict(CUBE, periodic=periodic, warp=warp), K, N, dt,
                      4, lambda o: o.bubble(amp=0.8, profile="sharp"))


def oracle_trajectory(q, q_init, precision, mesh, K, N, dt, nsteps, init, **phys):
    """The oracle advanced from its own initial state (which the GPU's must equal to
    1e-12) with the same step; q checked against it (oracle_checks bars)."""
    o = O.Oracle(*K, N, **mesh, **phys)
    q0 = init(o)
    assert np.abs(q_init - q0).max() <= 1e-12 * np.abs(q0).max()
    q_plain = o.steps(q0, dt, nsteps)
    if precision == "fp64":
        q_long = O.Oracle(*K, N, precision="long", **mesh, **phys).steps(q0, dt, nsteps)
        check_fp64(q, q_plain, q_long, what=(K, N, mesh))
    else:
        check_mixed(q, q0, q_plain, what=(K, N, mesh))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab_channel_with_coriolis(lib, precision):
    box = dict(lo=(0.0, 0.0, 0.0), hi=(40000e3, 6000e3, 30e3))
    kw = dict(mesh=box, f0=1e-4)
    whole, split, _ = pair(lib, (6, 3, 2), 4, 3, (1, 0, 0), 0.0, precision=precision, **kw)
    whole.init_channel()
    split.init_channel()
    q_init = split.get_state()
    dt = whole.cfl_dt(0.5)
    whole.step(dt, 3)
    split.step(dt, 2)
    split.step(dt, 1)
    q = split.get_state()
    assert np.array_equal(q, whole.get_state())
    oracle_trajectory(q, q_init, precision, dict(box, periodic=(1, 0, 0)), (6, 3, 2), 4, dt, 3,
                      lambda o: o.channel(), f0=1e-4)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab_step_graph_follows_dt_and_reconfiguration(lib, precision):
    # the captured step is replayed only for the time step and configuration it was
    # captured for: a new dt, a new background and new states all match the whole mesh
    K, N, parts, periodic, warp = CASES[1]
    whole, split, _ = pair(lib, K, N, parts, periodic, warp, precision=precision)
    for s in (whole, split):
        s.init_bubble(amp=0.8)
    dt = whole.cfl_dt(0.5)
    for s in (whole, split):
        s.step(dt, 2)
        s.step(dt, 2)
        s.step(0.5 * dt, 3)
    assert np.array_equal(split.get_state(), whole.get_state())
    for s in (whole, split):
        s.init_bubble(amp=0.3, profile="sharp")  # new state and background
        s.step(dt, 3)
    assert np.array_equal(split.get_state(), whole.get_state())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_split_face_launches_equal_the_stage(lib, precision):
    # the transport-agnostic sequence a process-per-slab caller runs (pack and
    # exchange, the faces that need no trace, the cut planes' faces, the volume
    # kernel with the stage update) equals the library's partitioned steps bitwise
    K, N, parts, periodic, warp = CASES[1]
    _, a, _ = pair(lib, K, N, parts, periodic, warp, precision=precision)
    _, b, _ = pair(lib, K, N, parts, periodic, warp, precision=precision)
    for s in (a, b):
        s.init_bubble(amp=0.8)
    dt = a.cfl_dt(0.5)
    a.step(dt, 2)
    for _ in range(2):
        for stage in range(5):
            b.exchange()
            for s in b.parts:
                s.launch(3, stage, dt)
                s.launch(4, stage, dt)
                s.launch(2, stage, dt)
    assert np.array_equal(a.get_state(), b.get_state())


def test_slab_calls_need_traces(lib):
    m = dict(CUBE, periodic=(1, 1, 0))
    s = lib.Solver(4, 2, 2, 3, part=(1, 3), **m)
    b, e, remote, n = s.partition_info()
    assert (b, e, remote, n) == (1, 3, (1, 1), 2 * 2 * 5 * 16)
    with pytest.raises(EsDgError):
        s.step(1e-3, 1)  # a slab steps only with its neighbours
    with pytest.raises(EsDgError):
        s.rhs(np.zeros(s.shape()))  # no traces registered yet
    s.close()
